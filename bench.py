#!/usr/bin/env python3
"""Benchmark of the LVQ search hot path on B300.

Workload (default): multi-means LVQ-4x8, 10,000,000 vectors of d = 768 drawn
from a 256-component Gaussian mixture (sigma 0.3, unit-normalised), 16
centring means fitted by k-means on a 100k sample, inner product.  One step
is one pass of the whole hot path over one batch of synthetic input:

  1. lvq_delete of 10,000 live slots and lvq_insert of 10,000 new vectors
     (mean assignment, centring, bounds, both code levels, slot reuse);
  2. lvq_search_exhaustive of a mix of uneven query batches (sizes {1, 4096}
     and 30 log-uniform draws in [1, 4096], concatenated into one launch),
     top-100 on the first level, re-ranked to top-10 with the residuals;
  3. lvq_search_candidates of 1,024 queries x 2,048 candidate ids (70% from
     the query's own component), top-50 re-ranked to top-10.

``value`` is first-level (query, vector) distances per second over the
whole step with inputs resident in HBM; ``e2e`` is the same through the C
ABI with the step's inputs copied from pinned host memory and its results
copied back inside the timed region.  The compressed database (3.9 GB of
codes) is larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "mlvq4x8-ip-10m-d768"
METRIC = "LVQ-4x8 distances/s & QPS@recall10 at 10M x 768"
UNIT = "distances/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one scan_mma launch over
# 2M rows with the bench's 12,716-query mix (ncu --set full, B300)
SCAN_MMA_DRAM_BYTES_2M = 2.029857e9 + 0.817906e9
# DRAM bytes (read + write) of one ID-gather launch of 1,024 queries x 2,048
# candidate ids, from an ncu capture of the same launch size at 2M rows (the
# launch's traffic depends on the candidates, not on the rows)
GATHER_DRAM_BYTES = 1.066799e9 + 4.035e6
# the same for the 5M x 96 ID-gather launch (8,192 queries x 2,048 ids)
GATHER2_C4_DRAM_BYTES = 1.060708e9 + 8.123e6
# first-level bytes of a database row at d = 768, 4 bits: codes, lower, step,
# mean id (IP reads no norm) and its live bit
ROW_BYTES = 384 + 4 + 4 + 4 + 1 / 8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="database size (default: the workload's)")
    ap.add_argument("--mix", default="full", choices=["full", "small"],
                    help="query mix: full = {1,4096} + 30 log-uniform in [1,4096]; small = 8 in [1,256]")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "fp16", "int16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the small-batch roofline leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-latency leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c2", action="store_true", help="skip the 1M x 768 fp16-vs-fp32 leg")
    ap.add_argument("--no-c4", action="store_true", help="skip the 5M x 96 ID-gather leg")
    ap.add_argument("--no-qps-recall", action="store_true", help="skip the k1 sweep for QPS at recall 0.9")
    ap.add_argument("--no-c5", action="store_true", help="skip the 20M x 200 streaming-serve leg")
    return ap.parse_args()


def query_mix(kind: str, seed: int):
    if kind == "small":
        return synth.log_uniform_sizes(8, 1, 256, seed)
    return np.concatenate([[1, 4096], synth.log_uniform_sizes(30, 1, 4096, seed)])


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons (200 ms)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks_file() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(units: float, seconds: float, world: int):
    """Whole-job units and the slowest rank's time (max over ranks)."""
    if world == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([units, seconds], dtype=torch.float64, device=dev)
    u = t[:1].clone()
    s = t[1:].clone()
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


# --------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the workload
# --------------------------------------------------------------------------

def cpu_baseline(mix, means, q_host, sample_rows=40_000, sample_queries=8, k1=100, k=10):
    import oracle as O
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    x = mix.rows(0, sample_rows)
    enc = O.encode(x, means, 4, 8)
    q = q_host[:sample_queries]
    t0 = time.perf_counter()
    O.search_exhaustive(enc, means, q, k1, k, O.IP)
    dt = time.perf_counter() - t0
    return {"value": sample_rows * sample_queries / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle brute-force search (first level over {sample_rows} rows of the workload, "
                      f"top-{k1}, two-level re-rank to top-{k}) for {sample_queries} queries; "
                      f"{dt:.2f} s; float64 decode + numpy/OpenBLAS"}


def serve_leg(st, mix, n, avoid, duration_s=6.0, rate=40.0, update_every_s=0.25, B_upd=10_000, seed=6006,
              warm_s=2.0):
    """p50/p99 latency of query requests served by the continuous-batching
    loop under mixed load: Poisson arrivals (rate per second) of batches of
    log-uniform size in [1, 4096] with k in {10, 100}, and every
    update_every_s an insert of B_upd new vectors plus a delete of B_upd
    live ones, all on the same store.  An untimed trace of warm_s seconds
    (other arrivals, the same mix) runs first: the first trace of a process
    on a freshly started GPU stalls for about a second in its first large
    search, a one-off that later traces do not show."""
    from paper_2402_02044_b300.serve import Server
    pool = mix.queries(8192)
    n_upd_max = int((duration_s + warm_s) / update_every_s) + 4
    cand = synth.choose(n, min(n, 3 * n_upd_max * B_upd), seed + 4)
    cand = cand[~np.isin(cand, np.fromiter(avoid, dtype=np.int64, count=len(avoid)))][:n_upd_max * B_upd]
    # every update batch is generated before the trace starts, so that the
    # client thread does no heavy work (and holds no interpreter lock) while
    # requests are in flight
    upd_rows = [mix.rows(u * B_upd, (u + 1) * B_upd, stream=13) for u in range(n_upd_max)]
    srv = Server(st, lanes=2, max_batch=1024, k1=100, kmax=100, precision="auto")
    used = [0]  # update batches used so far (each deletes its own slice of cand)

    def trace(secs, sd):
        count = max(1, int(secs * rate))
        t_arr = synth.poisson_arrivals(count, rate, sd)
        sizes = synth.log_uniform_sizes(count, 1, 4096, sd + 1)
        ks = np.where(synth.uniform_ints(count, 0, 1, sd + 2) == 0, 10, 100)
        offs = synth.uniform_ints(count, 0, 4096, sd + 3, tag=4)
        futs, upd = [], []
        t0 = time.perf_counter()
        next_upd = 0.0
        for i in range(count):
            while True:
                now = time.perf_counter() - t0
                u = used[0]
                if now >= next_upd and (u + 1) * B_upd <= len(cand) and u < len(upd_rows):
                    upd.append(srv.submit_delete(cand[u * B_upd:(u + 1) * B_upd]))
                    upd.append(srv.submit_insert(upd_rows[u]))
                    used[0] += 1
                    next_upd += update_every_s
                if now >= t_arr[i]:
                    break
                time.sleep(min(t_arr[i] - now, 0.0005))
            futs.append(srv.submit_query(pool[offs[i]:offs[i] + sizes[i]], int(ks[i])))
        for f in futs:
            f.result(timeout=120)
        failed = 0
        for f in upd:
            try:
                f.result(timeout=120)
            except Exception:
                failed += 1
        srv.drain()
        return failed

    trace(warm_s, seed + 100)
    srv.reset_stats()
    u0 = used[0]
    failed = trace(duration_s, seed)
    s = srv.stats_summary()
    srv.close()
    return {"requests": s.get("requests"), "p50_ms": s.get("p50_ms"), "p99_ms": s.get("p99_ms"),
            "mean_ms": s.get("mean_ms"), "qps": s.get("qps"), "epochs": s.get("epochs"),
            "offered": f"{rate:g} query batches/s (Poisson, sizes log-uniform 1..4096, k in {{10, 100}}) for "
                       f"{duration_s:g} s; every {update_every_s:g} s insert {B_upd} + delete {B_upd}; "
                       f"after an untimed {warm_s:g} s trace of the same mix",
            "update_batches": 2 * (used[0] - u0), "update_failures": failed, "lanes": 2, "max_batch": 1024,
            "precision": "auto", "slowest": s.get("slowest")}


def _timed(st, fn, reps=3, warm=1):
    """Mean wall milliseconds of fn() on the device (CUDA events) and the
    mean per-call milliseconds of each kernel kind the library timed."""
    import torch
    from paper_2402_02044_b300 import lvq as L
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    L.lvq_profile_enable(st.handle, True)
    L.lvq_profile_read(st.handle)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    prof = L.lvq_profile_read(st.handle)
    L.lvq_profile_enable(st.handle, False)
    return e0.elapsed_time(e1) / reps, {k: v[0] / reps for k, v in prof.items() if v[1]}


def _rel_err(q, ids, scores, enc, means, metric, level):
    """Largest |s - s_ref| / max(|s_ref|, ||q|| ||x^||) over the returned
    results, s_ref the oracle's float64 score of the returned id."""
    import oracle as O
    worst = 0.0
    for i in range(len(q)):
        sel = ids[i] >= 0
        if not sel.any():
            continue
        xh = O.decode(O.take(enc, ids[i][sel]), means, level)
        ref = O.score(q[i], xh, metric)[0]
        scl = np.maximum(np.abs(ref), np.linalg.norm(q[i].astype(np.float64)) * np.linalg.norm(xh, axis=1))
        worst = max(worst, float((np.abs(scores[i][sel].astype(np.float64) - ref) / scl).max()))
    return worst


def c2_leg(n=1_000_000, batches=(1, 64, 1024, 10_000), n_recall=100, k1s=(10, 20, 50, 100, 200)):
    """LVQ-4x8 inner product on 1M x 768 (one global mean): the float16
    tensor-core first level against the plain float32 one at each batch
    size (kernel time and distances/s), and, on n_recall queries against
    the oracle (encode, exact k-NN over the decoded vectors, two-level
    search): recall@10, agreement with the oracle's two-level result, the
    largest relative error of any returned score, and recall by k1."""
    import torch
    import oracle as O
    from paper_2402_02044_b300 import Store
    name = "lvq4x8-ip-1m-d768"
    mix = synth.mixture_for(name)
    x = mix.rows(0, n)
    mu = synth.sample_mean(x)[None]
    st = Store(x.shape[1], 4, 8, mu, "ip", n)
    for s0 in range(0, n, 1 << 20):
        st.insert(torch.from_numpy(x[s0:s0 + (1 << 20)]).cuda())
    q_host = mix.queries(max(batches))
    q_dev = torch.from_numpy(q_host).cuda()
    st.reserve(max(batches), max(k1s), 0)
    rows = []
    for B in batches:
        qb = q_dev[:B].contiguous()
        row = {"nq": B}
        for prec in ("fp16", "fp32"):
            ms, kern = _timed(st, lambda: st.search(qb, 10, 100, prec), reps=3 if B < 10_000 else 2)
            kind = "scan_mma" if prec == "fp16" else "scan_fp32"
            row[prec] = {"search_ms": ms, "scan_ms": kern.get(kind), "kernel": kind,
                         "distances_per_s": B * n / (kern[kind] / 1e3) if kern.get(kind) else None}
        row["fp32_over_fp16_scan_time"] = row["fp32"]["scan_ms"] / row["fp16"]["scan_ms"]
        rows.append(row)
    # against the oracle
    t0 = time.perf_counter()
    enc = O.encode(x, mu, 4, 8)
    qs = q_host[:n_recall]
    truth = O.ground_truth(enc, mu, qs, 10, O.IP)[0]
    cand1 = O.first_level_candidates(enc, mu, qs, max(k1s), O.IP)[0]
    t_oracle = time.perf_counter() - t0
    qs_dev = torch.from_numpy(qs).cuda()
    acc = {}
    for prec in ("fp16", "fp32"):
        fi, fs = (t.cpu().numpy() for t in st.first_level(qs_dev, 100, prec))
        gi, gs = (t.cpu().numpy() for t in st.search(qs_dev, 10, 100, prec))
        two = O.rerank(enc, mu, qs, cand1[:, :100], 10, O.IP)[0]
        acc[prec] = {"recall_at_10": O.recall_at_k(gi, truth, 10),
                     "agreement_with_oracle_two_level": O.recall_at_k(gi, two, 10),
                     "max_rel_err_first_level": _rel_err(qs, fi, fs, enc, mu, O.IP, 1),
                     "max_rel_err_reranked": _rel_err(qs, gi, gs, enc, mu, O.IP, 2)}
    by_k1 = []
    qb = q_dev[:batches[-1]].contiguous()
    for k1 in k1s:
        gi = st.search(qs_dev, 10, k1, "fp16")[0].cpu().numpy()
        two = O.rerank(enc, mu, qs, cand1[:, :k1], 10, O.IP)[0]
        ms, _ = _timed(st, lambda: st.search(qb, 10, k1, "fp16"), reps=2)
        by_k1.append({"k1": k1, "recall_at_10": O.recall_at_k(gi, truth, 10),
                      "oracle_recall_at_10": O.recall_at_k(two, truth, 10),
                      "agreement_with_oracle_two_level": O.recall_at_k(gi, two, 10),
                      "qps": len(qb) / (ms / 1e3), "qps_batch": len(qb)})
    ok = [r for r in by_k1 if r["recall_at_10"] >= 0.9]
    st.close()
    return {"workload": name, "n": n, "d": int(x.shape[1]), "metric": "ip", "k1": 100, "k": 10,
            "batches": rows, "vs_oracle": acc, "by_k1": by_k1,
            "qps_at_recall_0.9": ({"k1": ok[0]["k1"], "recall_at_10": ok[0]["recall_at_10"], "qps": ok[0]["qps"]}
                                  if ok else None),
            "oracle_sample": f"{n_recall} workload queries over all {n} vectors; oracle encode + search {t_oracle:.1f} s",
            "tolerance": {"fp16_first_level": 2e-3, "fp32": 1e-5,
                          "scale": "max(|s|, ||q|| ||x^||)"}}


def c4_leg(n=5_000_000, nq=8192, C=2048, k1=50, k=10):
    """ID-gather form on 5M x 96 L2 LVQ-4x8: 8,192 queries x 2,048 candidate
    ids (70 % from the query's own mixture component, 30 % uniform), top-50
    on the first level re-ranked to top-10; the gather kernel against the
    measured HBM copy bandwidth."""
    import torch
    from paper_2402_02044_b300 import Store
    name = "gather-lvq4x8-l2-5m-d96"
    w = synth.WORKLOADS[name]
    mix = synth.mixture_for(name)
    mu = synth.running_mean(mix, n)[None]
    st = Store(w["d"], 4, 8, mu, "l2", n)
    for s0 in range(0, n, 1 << 20):
        st.insert(torch.from_numpy(mix.rows(s0, min(n, s0 + (1 << 20)))).cuda())
    lab = mix.labels(0, n)
    qh, qlab = mix.rows(0, nq, stream=3, with_labels=True)
    cand = synth.candidate_lists(lab, qlab, C, w["frac_own"], seed=4004)
    qd, cd = torch.from_numpy(qh).cuda(), torch.from_numpy(cand).cuda()
    st.reserve(nq, k1, C)
    ms, kern = _timed(st, lambda: st.search_candidates(qd, cd, k, k1), reps=5)
    row1 = ((w["d"] * 4 // 8) + 15) // 16 * 16
    per_cand = row1 + 16 + 8   # the record (codes, then l, D, ||x^||^2, mean id) and the candidate id
    g_ms = kern.get("gather")
    peak = peaks_file().get("hbm_gbs")
    gbs = nq * C * per_cand / g_ms / 1e6 if g_ms else None
    st.close()
    return {"workload": name, "n": n, "d": w["d"], "metric": "l2", "queries": nq, "candidates": C, "k1": k1, "k": k,
            "search_ms": ms, "kernel_ms": kern, "qps": nq / (ms / 1e3),
            "gather_roofline": {"kernel": "gather2_kernel", "bound": "hbm", "bytes_per_candidate": per_cand,
                                "algorithmic_bytes_per_launch": nq * C * per_cand, "kernel_ms": g_ms,
                                "achieved": gbs, "peak": peak, "unit": "GB/s",
                                "frac": gbs / peak if gbs and peak else None,
                                "traffic": GATHER2_C4_DRAM_BYTES if (n, nq, C) == (5_000_000, 8192, 2048) else None,
                                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak else None}}


def c5_leg(n=20_000_000, steps=4, step_s=1.5, frac=0.01, n_recall=100, seed=5005):
    """Streaming serve with distribution shift: a 20M-slot LVQ-4x8 L2 store
    of d = 200 filled from 128 mixture components (centred by the mean of
    that fill, fixed thereafter); each step deletes 1 % of the live slots and
    inserts 1 % new vectors from 8 components unseen at the fill (encoded on
    the device into reused slots) while a Poisson stream of query batches
    (sizes log-uniform in [1, 4096], k in {10, 100}) at 0.7 of the measured
    single-stream capacity is served; p50 / p99 latency, QPS, and after each
    step recall@10 of 100 queries from the live mixture against the exact
    top-10 of the decoded vectors (float64 on the GPU, checked against the
    oracle by the tests)."""
    import torch
    from paper_2402_02044_b300 import Store
    from paper_2402_02044_b300 import robustness as R
    from paper_2402_02044_b300.serve import Server
    name = "stream-lvq4x8-l2-20m-d200"
    w = synth.WORKLOADS[name]
    mix = synth.mixture_for(name)
    old = np.arange(w["comps"])
    new = np.arange(w["comps"], w["comps"] + w["new_comps"])
    t0 = time.perf_counter()
    chunk = 1 << 21
    parts, acc = [], np.zeros(w["d"], np.float64)
    for s0 in range(0, n, chunk):
        xs = mix.rows(s0, min(n, s0 + chunk), comps=old)
        acc += xs.astype(np.float64).sum(0)
        parts.append(torch.from_numpy(xs).cuda())
    mu = (acc / n).astype(np.float32)[None]
    n_step = int(frac * n)
    cap = n + 2 * n_step          # deletes are held one boundary before reuse
    st = Store(w["d"], 4, 8, mu, "l2", cap)
    for xs in parts:
        st.insert(xs)
    del parts
    torch.cuda.synchronize()
    t_fill = time.perf_counter() - t0
    live = np.zeros(cap, bool)
    live[:n] = True
    pool = mix.queries(8192, comps=np.concatenate([old, new]))
    # single-stream capacity: batches of the trace's size distribution, one at a time
    probe_sizes = synth.log_uniform_sizes(16, 1, 4096, seed + 9)
    qd = torch.from_numpy(pool).cuda()
    st.reserve(4096, 100, 0)
    for b in probe_sizes[:3]:
        st.search(qd[:b].contiguous(), 10, 100, "auto")
    torch.cuda.synchronize()
    tc = time.perf_counter()
    for b in probe_sizes:
        st.search(qd[:b].contiguous(), 10, 100, "auto")
    torch.cuda.synchronize()
    per_batch = (time.perf_counter() - tc) / len(probe_sizes)
    rate = 0.7 / per_batch
    srv = Server(st, lanes=2, max_batch=1024, k1=100, kmax=100, precision="auto")
    count = max(1, int(steps * step_s * rate))
    t_arr = synth.poisson_arrivals(count, rate, seed)
    sizes = synth.log_uniform_sizes(count, 1, 4096, seed + 1)
    ks = np.where(synth.uniform_ints(count, 0, 1, seed + 2) == 0, 10, 100)
    offs = synth.uniform_ints(count, 0, 4096, seed + 3, tag=4)
    ins_rows = [mix.rows(u * n_step, (u + 1) * n_step, stream=7, comps=new) for u in range(steps)]
    g = np.random.default_rng(seed)
    recalls, futs, upd = [], [], []
    qr = torch.from_numpy(mix.rows(0, n_recall, stream=19, comps=np.concatenate([old, new]))).cuda()
    t_start = time.perf_counter()
    paused = 0.0  # time spent measuring recall between steps (the arrival clock stops)
    i = 0
    for u in range(steps):
        dele = np.sort(g.choice(np.nonzero(live)[0], n_step, replace=False))
        live[dele] = False
        upd.append(srv.submit_delete(dele))
        fi = srv.submit_insert(ins_rows[u])
        upd.append(fi)
        t_end = (u + 1) * step_s
        while i < count and t_arr[i] < t_end:
            now = time.perf_counter() - t_start - paused
            if now < t_arr[i]:
                time.sleep(min(t_arr[i] - now, 0.0005))
                continue
            futs.append(srv.submit_query(pool[offs[i]:offs[i] + sizes[i]], int(ks[i])))
            i += 1
        ids = fi.result(timeout=300)
        live[ids] = True
        # recall once this step's updates are visible and its queries done;
        # the arrival clock stops meanwhile, so the next step's requests are
        # not released all at once
        tp = time.perf_counter()
        for f in futs:
            f.result(timeout=300)
        srv.drain(timeout=300)
        truth = R.decoded_truth(st, qr, 10, level=2, n_rows=cap, chunk=1 << 21)
        got, _ = st.search(qr, 10, 100, "auto")
        recalls.append(R.recall(got, truth, 10))
        paused += time.perf_counter() - tp
    failed = 0
    for f in upd:
        try:
            f.result(timeout=300)
        except Exception:
            failed += 1
    s = srv.stats_summary()
    srv.close()
    st.close()
    return {"workload": name, "slots": cap, "live": int(live.sum()), "d": w["d"], "metric": "l2",
            "steps": steps, "per_step": f"delete {n_step} + insert {n_step} (8 unseen components)",
            "offered_batches_per_s": rate, "single_stream_ms_per_batch": per_batch * 1e3,
            "requests": s.get("requests"), "p50_ms": s.get("p50_ms"), "p99_ms": s.get("p99_ms"),
            "mean_ms": s.get("mean_ms"), "qps": s.get("qps"), "recall_at_10_by_step": recalls,
            "recall_truth": "exact top-10 over the decoded two-level vectors (float64), 100 queries",
            "update_failures": failed, "fill_s": t_fill, "slowest": s.get("slowest")}


def qps_at_recall(st, q_dev, q_recall, sizes_total, k1s=(50, 100, 200, 512), target=0.9):
    """Recall@10 of the two-level search on the benchmark store against the
    exact top-10 of its decoded vectors (float64 on the GPU, checked against
    the oracle by the tests) for each k1, and the queries per second of the
    benchmark's query mix at the smallest k1 that reaches the target."""
    import torch
    from paper_2402_02044_b300 import robustness as R
    truth = R.decoded_truth(st, q_recall, 10, level=2, n_rows=None)
    out = []
    for k1 in k1s:
        gi, _ = st.search(q_recall, 10, k1, "auto")
        ms, _ = _timed(st, lambda: st.search(q_dev, 10, k1, "auto"), reps=1)
        out.append({"k1": k1, "recall_at_10": R.recall(gi, truth, 10), "qps": sizes_total / (ms / 1e3),
                    "search_ms": ms})
    ok = [r for r in out if r["recall_at_10"] >= target]
    res = {"by_k1": out, "target": target, "queries": len(q_recall),
           "truth": "exact top-10 over the decoded two-level vectors (float64)",
           "note": None if ok else ("recall@10 0.9 is not reached at k1 <= %d on this mixture (first-level "
                                    "candidates are capped at 512 per query); QPS is given per k1" % max(k1s))}
    if ok:
        r = ok[0]
        res.update(k1=r["k1"], recall_at_10=r["recall_at_10"], qps=r["qps"], search_ms=r["search_ms"])
    torch.cuda.synchronize()
    return res


def run_reference(args):
    """--impl reference: the oracle timed on the host cores, same metric."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    w = synth.WORKLOADS[WORKLOAD]
    mix = synth.mixture_for(WORKLOAD)
    means = synth.kmeans_means(mix.rows(0, 20_000, stream=5), w["n_means"], seed=3003, iters=10)
    q = mix.queries(16)
    times = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(mix, means, q, sample_rows=20_000, sample_queries=4)
        if i >= args.warmup:
            times.append(r)
        base = r
    vals = [r["value"] for r in times] or [base["value"]]
    value = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": w["n"], "d": w["d"], "n_means": w["n_means"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    world, rank, local = dist_setup()
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2402_02044_b300 import build
    build.build()
    from paper_2402_02044_b300 import Store
    from paper_2402_02044_b300 import lvq as L

    w = synth.WORKLOADS[WORKLOAD]
    n = args.n or w["n"]
    d = w["d"]
    mix = synth.mixture_for(WORKLOAD)
    t_setup = time.time()
    sample = mix.rows(0, min(w["kmeans_sample"], n), stream=5)
    means = synth.kmeans_means(sample, w["n_means"], seed=3003, iters=25)
    B_upd = 10_000
    steps_total = args.warmup + 2 * args.steps
    st = Store(d, 4, 8, means, "ip", n + 100_000)  # spare slots for the serving leg's inserts
    chunk = 1 << 20
    for s in range(0, n, chunk):
        xs = torch.from_numpy(mix.rows(s, min(n, s + chunk))).cuda()
        st.insert(xs)
    torch.cuda.synchronize()
    assert st.stats() == n
    # queries
    sizes = query_mix(args.mix, 4003)
    nq = int(sizes.sum())
    q_host = mix.queries(nq)
    q_dev = torch.from_numpy(q_host).cuda()
    # ID-gather batch
    nq_g, C = 1024, 2048
    lab_db = mix.labels(0, n)
    qg_host, qg_lab = mix.rows(0, nq_g, stream=3, with_labels=True)
    cand_host = synth.candidate_lists(lab_db, qg_lab, C, 0.7, seed=4004)
    qg_dev = torch.from_numpy(qg_host).cuda()
    cand_dev = torch.from_numpy(cand_host).cuda()
    # per-step update batches: delete initially filled slots, insert fresh vectors
    g = np.random.default_rng(7000 + rank)
    del_host = [np.sort(g.choice(n, B_upd, replace=False)).astype(np.int64) for _ in range(steps_total)]
    # keep the delete sets disjoint from each other's re-inserted slots: draw
    # every step's ids from slots that are still original
    used = set()
    for i in range(steps_total):
        s_ = [v for v in del_host[i].tolist() if v not in used]
        while len(s_) < B_upd:
            extra = int(g.integers(0, n))
            if extra not in used and extra not in s_:
                s_.append(extra)
        del_host[i] = np.array(sorted(s_), dtype=np.int64)
        used.update(s_)
    ins_host = [mix.rows(i * B_upd, (i + 1) * B_upd, stream=7) for i in range(steps_total)]
    del_dev = [torch.from_numpy(a).cuda() for a in del_host]
    ins_dev = [torch.from_numpy(a).cuda() for a in ins_host]
    precision = args.precision
    st.reserve(nq, 100, C)
    # the tensor-core scan's tile shape for this batch, chosen by the autotuner
    # (query-tile widths 64 and 128, timed with the library's own events)
    tuning = None
    if not args.no_autotune and precision in ("auto", "fp16"):
        from paper_2402_02044_b300 import autotune
        best = autotune.autotune(st, q_dev, n, sizes=(nq,), k1=100, reps=1, widths=(64, 128), ctas_opts=(0,))
        tuning = autotune.tuning_for(best, nq)
        st.set_tuning(**tuning)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup

    def step(i, qd, qgd, cd, dd, xd):
        st.delete(dd)
        st.insert(xd)
        ids, sc = st.search(qd, 10, 100, precision)
        gi, gs = st.search_candidates(qgd, cd, 10, 50)
        return ids, sc, gi, gs

    for i in range(args.warmup):
        step(i, q_dev, qg_dev, cand_dev, del_dev[i], ins_dev[i])
    torch.cuda.synchronize()

    # timed region (device-resident inputs)
    clocks = ClockSampler(local)
    clocks.start()
    L.lvq_profile_enable(st.handle, True)
    L.lvq_profile_read(st.handle)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(args.steps):
        j = args.warmup + i
        step(j, q_dev, qg_dev, cand_dev, del_dev[j], ins_dev[j])
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = L.lvq_profile_read(st.handle)
    L.lvq_profile_enable(st.handle, False)
    t_dev = ev0.elapsed_time(ev1) / 1e3
    n_live = st.stats()
    dist_per_step = nq * n_live + nq_g * C
    units, t_max = aggregate(dist_per_step * args.steps, t_dev, world)
    value = units / t_max
    qps = (nq + nq_g) * args.steps * world / t_max

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
        q_pin, qg_pin, cand_pin = pin(q_host), pin(qg_host), pin(cand_host)
        del_pin = [pin(a) for a in del_host]
        ins_pin = [pin(a) for a in ins_host]
        out_pin = [torch.empty((nq, 10), dtype=torch.int64).pin_memory(),
                   torch.empty((nq, 10), dtype=torch.float32).pin_memory(),
                   torch.empty((nq_g, 10), dtype=torch.int64).pin_memory(),
                   torch.empty((nq_g, 10), dtype=torch.float32).pin_memory()]
        h2d = q_host.nbytes + qg_host.nbytes + cand_host.nbytes + del_host[0].nbytes + ins_host[0].nbytes
        d2h = sum(t.numel() * t.element_size() for t in out_pin)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            j = args.warmup + args.steps + i
            qd = q_pin.cuda(non_blocking=True)
            qgd = qg_pin.cuda(non_blocking=True)
            cd = cand_pin.cuda(non_blocking=True)
            dd = del_pin[j].cuda(non_blocking=True)
            xd = ins_pin[j].cuda(non_blocking=True)
            res = step(j, qd, qgd, cd, dd, xd)
            for o, r in zip(out_pin, res):
                o.copy_(r, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        t_e2e = e0.elapsed_time(e1) / 1e3
        u2, t2 = aggregate(dist_per_step * args.steps, t_e2e, world)
        e2e = {"value": u2 / t2, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # the autotuned tile width was for the step's 12,716-query batch; the
    # other legs on this store pick their tiles by batch size
    if tuning:
        st.set_tuning()
    # small batches: the integer scan against the HBM roofline
    bytes_per_row = ROW_BYTES
    hbm_peak = peaks_file().get("hbm_gbs")
    small = None
    if not args.no_small:
        small = []
        for nqs in (1, 2, 4, 8, 16, 32, 64):
            qs = q_dev[:nqs].contiguous()
            for _ in range(3):
                st.search(qs, 10, 100, "auto")
            torch.cuda.synchronize()
            L.lvq_profile_enable(st.handle, True)
            L.lvq_profile_read(st.handle)
            reps = 20
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            for _ in range(reps):
                st.search(qs, 10, 100, "auto")
            s1.record()
            torch.cuda.synchronize()
            p2 = L.lvq_profile_read(st.handle)
            L.lvq_profile_enable(st.handle, False)
            kind = max(("scan_small", "scan_mma", "scan_fp32"), key=lambda kk: p2[kk][1])
            kms = p2[kind][0] / max(p2[kind][1], 1)
            gbs = n_live * bytes_per_row / kms / 1e6
            small.append({"nq": nqs, "kernel": kind, "kernel_ms": kms, "hbm_gbs": gbs, "peak_gbs": hbm_peak,
                          "frac": gbs / hbm_peak if hbm_peak else None,
                          "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_peak else None,
                          "search_ms": s0.elapsed_time(s1) / reps,
                          "kernel_ms_per_search": {kk: v[0] / reps for kk, v in p2.items() if v[1]}})

    serve = None
    if not args.no_serve:
        serve = serve_leg(st, mix, n, used)
    qr = None
    if not args.no_qps_recall and rank == 0:
        qr = qps_at_recall(st, q_dev, q_dev[:100].contiguous(), nq)
    c2 = None if args.no_c2 or rank != 0 else c2_leg()
    c4 = None if args.no_c4 or rank != 0 else c4_leg()
    c5 = None if args.no_c5 or rank != 0 else c5_leg()

    # roofline of the dominant kernel
    scan_kind = "scan_mma" if prof["scan_mma"][1] else "scan_fp32"
    scan_ms, scan_launches = prof[scan_kind]
    peaks = peaks_file()
    flops_per_launch = 2.0 * nq * n_live * d
    bytes_per_launch = n_live * ROW_BYTES
    per_launch_s = scan_ms / 1e3 / max(scan_launches, 1)
    if scan_kind == "scan_mma":
        achieved = flops_per_launch / per_launch_s / 1e12
        peak = peaks.get("bf16_tflops_sustained") or 1400.0
        # DRAM bytes of one launch: an ncu capture of this kernel at 2M rows
        # (dram__bytes_read.sum + dram__bytes_write.sum, same query mix),
        # scaled by the rows (jobs and their code reads grow with the rows)
        traffic = SCAN_MMA_DRAM_BYTES_2M * n_live / 2e6 if nq == 12716 else None
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": "ncu capture at 2M rows scaled by rows" if traffic else None,
                "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops_sustained; fp16 rate = bf16 rate)"
                if "bf16_tflops_sustained" in peaks else "fallback"}
    else:
        achieved = flops_per_launch / per_launch_s / 1e12
        mhz = clk.get("sm_mhz") or 1900.0
        peak = 148 * 128 * 2 * mhz * 1e6 / 1e12   # FP32 FMA lanes x 2 flops x clock
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x median SM clock"}
    # the ID-gather kernel of the step (candidate ids, codes and per-row
    # constants of every candidate, re-rank reads not counted)
    g_ms = prof["gather"][0] / max(prof["gather"][1], 1)
    g_bytes = nq_g * C * (384 + 16 + 8)  # the record (codes and trailer) and the candidate id
    gather_roof = {"kernel": "gather_kernel", "kernel_ms": g_ms, "algorithmic_bytes_per_launch": g_bytes,
                   "hbm_gbs": g_bytes / g_ms / 1e6 if g_ms else None, "peak_gbs": peaks.get("hbm_gbs"),
                   "frac": g_bytes / g_ms / 1e6 / peaks["hbm_gbs"] if g_ms and peaks.get("hbm_gbs") else None,
                   "traffic": GATHER_DRAM_BYTES if (nq_g, C) == (1024, 2048) else None}
    roof["kernel"] = scan_kind
    roof["algorithmic_bytes_per_launch"] = bytes_per_launch
    roof["hbm_gbs_equiv"] = bytes_per_launch / per_launch_s / 1e9
    launches = sum(c for _, c in prof.values())

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16xf16->f32 (first level), f32 (encode, re-rank)" if scan_kind == "scan_mma" else "f32",
            "data": "synthetic (seeded Gaussian mixture; stands in for the paper's datasets)",
            "config": {"workload": WORKLOAD, "n": n, "d": d, "bits": "4x8", "n_means": w["n_means"],
                       "metric": "ip", "queries_per_step": int(nq), "query_batches": [int(v) for v in sizes],
                       "k1": 100, "k": 10, "gather_queries": nq_g, "gather_candidates": C,
                       "updates_per_step": B_upd, "l2_flush": "not needed: 3.9 GB of codes > 126 MB L2",
                       "precision": precision, "autotuned_tiles": tuning},
            "qps": qps, "recall_at_10": None, "small_batch": small, "serve": serve, "gather_roofline": gather_roof,
            "qps_at_recall": qr, "c2_fp16_vs_fp32": c2, "c4_id_gather": c4, "c5_streaming": c5,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "e2e": e2e,
            "setup_s": t_setup}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(mix, means, q_host)
    if qr:
        line["recall_at_10"] = next((r["recall_at_10"] for r in qr["by_k1"] if r["k1"] == 100), None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    st.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
