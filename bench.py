#!/usr/bin/env python3
"""Throughput of PLDS batch updates (edge updates/s at batch 1e6) on one GB300.

Workload: R-MAT scale 20, (a,b,c,d) = (.57,.19,.19,.05), edge factor 16,
symmetrised and deduplicated (~15.7M undirected int32 edges on 2^20 vertices),
delta = 0.4, lambda = 3.  A step is one batch of 10^6 edge updates through the
whole hot path (preprocessing, adjacency, counters, level rounds) followed by a
coreness query of every vertex.  The step stream cycles Ins (all edges from
empty, shuffled, batches of 10^6) then Del (all edges, a second shuffle).
The graph state (adjacency pool, level and counter arrays, ~1 GB) is larger
than L2, so no explicit L2 flush is done between steps.

The same line carries the Ins/Del/Mix protocols (Algorithm 2, PLDSOpt's group
size, the filter+sort insertion variant) and the two system forms on their own
workloads: serving (a device-resident request loop) and batched (512 graphs in
one launch per round), each with its clocks and a CPU baseline of the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
                  [--form plain|serving|batched|large] [--no-forms]

N > 1 (under torchrun) runs N independent replicas of the plain form (a single
graph's level rounds do not shard); value = all ranks' updates / max time.  With
--form batched the 512 graphs are split over the ranks by a greedy size balance
(no data-path collective).  --impl reference times the sequential CPU oracle on
the host cores on bounded samples of the same stream.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2106_03824_gb300 import workloads as W  # noqa: E402

METRIC = "edge updates/s at batch 1e6 (Ins/Del/Mix)"
UNIT = "updates/s"

# dram bytes / executed algorithmic bytes of the batch kernel, from the ncu capture
# summarised in profiles/ (kernel source hash at capture time); traffic is
# reported as null when the kernel source has changed since.
# DRAM bytes per algorithmic byte, from an ncu counter capture of the timed steps'
# kernels (profiles/traffic_rmat20_B1e6.md); valid only for the kernel sources it was
# taken on (kernel_sha), otherwise `traffic` is reported as null.
NCU_TRAFFIC = {"kernel_sha": "c837abe3941c36e1", "rounds_dram_per_algo_byte": 0.670,
               "batch_dram_per_algo_byte": 2.158,
               "capture": "ncu DRAM counters of every kernel of the timed steps of the R-MAT 20 stream, "
                          "Ins 14-15 and Del 0-1 (profiles/traffic_rmat20_B1e6.md)"}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2106_03824_gb300" / "csrc").iterdir()):
        if f.suffix in (".cu", ".cuh", ".h", ".cpp"):
            h.update(f.read_bytes())
    return h.hexdigest()[:16]


def whole_job(dist, updates: float, seconds: float, device: str):
    """The whole-job figures of a multi-rank run: the updates of every rank and the
    slowest rank's time (one collective each; the identity without a process
    group).  Returns (total updates, max seconds)."""
    if dist is None:
        return updates, seconds
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(u.item()), float(t.item())


def shard_graphs(sizes, parts: int):
    """Greedy size balance of independent graphs over `parts` ranks (or processes):
    graphs in decreasing size, each to the part with the least total so far (the
    lowest index on ties).  Returns each part's graph indices, ascending."""
    load = [0] * parts
    out = [[] for _ in range(parts)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        p = min(range(parts), key=lambda q: (load[q], q))
        out[p].append(i)
        load[p] += sizes[i]
    return [sorted(x) for x in out]


def algo_bytes(s: dict, kind: str) -> int:
    """Algorithmic bytes of the work one batch-kernel launch executed: 8 B per
    submitted edge; 64 B per applied update (2 probes + 2 slot writes of 4 B, 6
    counter read-modify-writes of 8 B); 4 B per level change; 8 B (id + level) per
    neighbour a move must examine -- an insertion move its up-neighbours
    (up_visits), a deletion move all its neighbours (visits); 8 B per neighbour read
    by a desire-level evaluation.  Rounds the kernel skipped (counted, not run) are
    left out."""
    moved = (s["up_visits"] - s["skipped_up_visits"]) if kind == "ins" else (s["visits"] - s["skipped_visits"])
    return (8 * s["submitted"] + 64 * s["valid"] + 4 * (s["moves"] - s["skipped_moves"]) + 8 * moved
            + 8 * s["dl_visits"])


def algo_bytes_degree(s: dict) -> int:
    """The same work under the scope table's per-unit figures: per move 4 B (level)
    + 8 B per neighbour of the mover (its degree) + 8 B per neighbour whose counter
    the move changed (affected); per desire-level evaluation 8 B per neighbour;
    per valid update 64 B; per submitted edge 8 B.  Executed rounds only."""
    return (8 * s["submitted"] + 64 * s["valid"] + 4 * (s["moves"] - s["skipped_moves"])
            + 8 * (s["visits"] - s["skipped_visits"]) + 8 * s["affected"] + 8 * s["dl_visits"])


def algo_bytes_steps(s: dict) -> int:
    """The part of algo_bytes that the step kernels before the level rounds do: 8 B
    per submitted edge, 64 B per applied update.  The rest (level writes, neighbour
    examinations, desire-level scans) is the rounds kernel's."""
    return 8 * s["submitted"] + 64 * s["valid"]


def algo_bytes_with_skipped(s: dict, kind: str) -> int:
    """algo_bytes with the skipped rounds counted as Algorithm 2 would run them (the
    bytes of the method's own level-by-level schedule; not a bandwidth figure)."""
    moved = s["up_visits"] if kind == "ins" else s["visits"]
    return 8 * s["submitted"] + 64 * s["valid"] + 4 * s["moves"] + 8 * moved + 8 * s["dl_visits"]


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def host_cpu() -> dict:
    """The host CPU's model (lscpu) and its logical core count."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model or platform.processor() or platform.machine(), "logical_cores": os.cpu_count(),
            "arch": platform.machine()}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def pct(x, q):
    return float(np.percentile(np.asarray(x, dtype=np.float64), q)) if len(x) else None


def make_stream(scale: int, batch: int, seed: int = 1):
    e = W.rmat(scale, 16, seed=seed)
    ins = W.shuffled(e, 11)
    dele = W.shuffled(e, 12)
    steps = [("ins", s, min(s + batch, e.shape[0])) for s in range(0, e.shape[0], batch)]
    steps += [("del", s, min(s + batch, e.shape[0])) for s in range(0, e.shape[0], batch)]
    return e, ins, dele, steps


def run_protocols(P, n, e, ins_d, del_d, mix_batches=10, seed=3, levels_per_group=0,
                  sizes=(1_000_000, 100_000), jump=False):
    """The experiments' Ins / Del / Mix protocols on the same graph, plain form,
    device-resident inputs: Ins all edges from empty and Del them all, in batches of
    1e6 and 1e5; Mix = 50/50 insert/delete batches of 1e6 on a 90 %-loaded graph
    (untimed preload).  Per protocol: updates/s (submitted and valid) over the whole
    sequence, the p50/p99 of the per-batch latency (CUDA events on the handle's
    stream between consecutive synchronous calls: submit to completion, no host
    staging since the batches are on the device), and the rounds and moves."""
    import torch

    def timed(g, calls):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
        upd, sts = 0, []
        torch.cuda.synchronize()
        evs[0].record()
        for i, (fn, b) in enumerate(calls):
            fn(b)
            upd += b.shape[0]
            evs[i + 1].record()
            sts.append(g.stats())
        torch.cuda.synchronize()
        lat = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(calls))]
        tot = evs[0].elapsed_time(evs[-1])
        return {"updates_per_s": upd / (tot / 1e3), "batches": len(calls),
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
                "valid_updates_per_s": sum(x["valid"] for x in sts) / (tot / 1e3),
                "rounds": sum(x["rounds"] for x in sts), "moves": sum(x["moves"] for x in sts),
                "rounds_run": sum(x["rounds"] - x["skipped_rounds"] for x in sts)}

    out = {}
    for B in sizes:
        tag = "1e6" if B == 1_000_000 else "1e5"
        g = P.PLDS(n, levels_per_group=levels_per_group, jump=jump)
        out[f"ins_{tag}"] = timed(g, [(g.insert, ins_d[s:s + B]) for s in range(0, ins_d.shape[0], B)])
        if B == sizes[0] and levels_per_group == 0 and not jump:
            # the static approximate k-core (Algorithm 6) of the loaded graph
            d = torch.empty(n, dtype=torch.float64, device="cuda")
            g.static_coreness(1.0, out=d)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st = g.static_coreness(1.0, out=d)
            e1.record()
            torch.cuda.synchronize()
            out["static_kcore"] = {"eps_prime": 1.0, "ms": e0.elapsed_time(e1), **st,
                                   "edges_per_s": int(e.shape[0]) / (e0.elapsed_time(e1) / 1e3)}
        out[f"del_{tag}"] = timed(g, [(g.delete, del_d[s:s + B]) for s in range(0, del_d.shape[0], B)])
        g.close()
    pre, mixes = W.mix_stream(e, 1_000_000, mix_batches, load=0.9, seed=seed)
    g = P.PLDS(n, levels_per_group=levels_per_group, jump=jump)
    pre_d = torch.from_numpy(pre).cuda()
    for s in range(0, pre_d.shape[0], 1_000_000):
        g.insert(pre_d[s:s + 1_000_000])
    calls = []
    for a, b in mixes:  # a mixed batch: its insertion half, then its deletion half
        calls.append((g.insert, torch.from_numpy(a).cuda()))
        calls.append((g.delete, torch.from_numpy(b).cuda()))
    m = timed(g, calls)
    g.close()
    m["batches"] = len(mixes)
    m["note"] = "p50/p99 over the halves (each half is one call)"
    out["mix_1e6"] = m
    return out


def cpu_sample(scale, ins, sample_batch=500_000):
    """The oracle (as it stands, 1 core) on a bounded prefix of the stream's first batch."""
    from oracle import oracle as O
    o = O.OraclePLDS(1 << scale)
    b = ins[:sample_batch]
    t0 = time.perf_counter()
    o.insert(b)
    dt = time.perf_counter() - t0
    return {"value": b.shape[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"first {b.shape[0]} edges of the first Ins batch of the same R-MAT scale-{scale} "
                      f"stream, applied as one batch to the empty graph ({dt:.1f} s on 1 host core; the "
                      f"full 10^6-edge batch takes minutes)"}


def plain_config(args, n: int, m: int, world: int, batch: int | None = None) -> dict:
    """The workload of the default (plain-form) bench line at `batch` edges a step
    (default: args.batch); the reference arm states the batch it ran."""
    b = args.batch if batch is None else batch
    return {"workload": f"rmat{args.scale}_ef16_B{b:.0e}_ins_del_cycle".replace("+0", ""),
            "graph": f"R-MAT scale {args.scale}, (.57,.19,.19,.05), edge factor 16, symmetrised, deduplicated",
            "n": n, "m": m, "batch": b, "delta": 0.4, "lambda": 3,
            "stream": "Ins all edges from empty, then Del all edges (cyclic)",
            "form": "plain: one synchronous launch sequence per batch",
            "l2": "no flush: graph state (~1 GB adjacency + arrays) is larger than the 129 MB L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    e, ins, dele, steps = make_stream(args.scale, args.batch)
    from oracle import oracle as O
    o = O.OraclePLDS(1 << args.scale)
    b = args.ref_batch
    pos = 0

    def step():
        nonlocal pos
        if pos >= ins.shape[0]:
            pos = 0
        chunk = ins[pos:pos + b]
        o.insert(chunk)
        pos += chunk.shape[0]
        return chunk.shape[0]

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    upd = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = upd / dt
    cfg = plain_config(args, 1 << args.scale, int(e.shape[0]), int(os.environ.get("WORLD_SIZE", "1")), batch=b)
    cfg["native_arm_batch"] = args.batch
    cfg["stream"] = "Ins edges of the same stream from empty (the oracle takes minutes per 10^6-edge batch)"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
                             "sample": f"the sequential CPU oracle as it stands, on 1 host core: {args.steps} "
                                       f"consecutive Ins batches of {b} edges of the same stream from the empty "
                                       f"graph, after {args.warmup} warm-up batches (a full {args.batch}-edge "
                                       f"batch takes the oracle minutes)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _batched_graph(args):
    """Graph i of the batched workload and its round batches, from its own seed:
    n log-uniform in [1e3,1e5], Chung-Lu exponent U[2.1,2.8], average degree
    U[4,32]; half of its edges preloaded (shuffled), then `rounds` mixed batches,
    each inserting 0.5-5 % of its edges taken from the absent pool and deleting as
    many present ones; the pools are queues, so a deleted edge can come back later."""
    i, rounds, seed = args
    rng = np.random.default_rng((seed, i))
    n = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
    e = W.chung_lu(n, int(n * rng.uniform(4, 32) / 2), rng.uniform(2.1, 2.8), seed=seed * 100003 + i)
    e = e[rng.permutation(e.shape[0])]
    half = e.shape[0] // 2
    present, absent = e[:half], e[half:]
    rs = []
    for _ in range(rounds):
        k = max(1, int(rng.uniform(0.005, 0.05) * e.shape[0]))
        k = min(k, present.shape[0], absent.shape[0])
        ins, dele = absent[:k], present[:k]
        rs.append((np.ascontiguousarray(ins), np.ascontiguousarray(dele)))
        absent = np.concatenate([absent[k:], dele])
        present = np.concatenate([present[k:], ins])
    return n, np.ascontiguousarray(e[:half]), rs


def make_batched(graphs: int, rounds: int, seed: int = 7, procs: int | None = None):
    """The batched form's workload: `graphs` independent graphs (see _batched_graph),
    generated in parallel host processes (spawned: safe after the GPU is in use).
    Returns (ns, preloads, rounds[r][i] = (insertions, deletions))."""
    import multiprocessing as mp
    procs = procs or min(graphs, os.cpu_count() or 1)
    jobs = [(i, rounds, seed) for i in range(graphs)]
    if procs > 1:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_batched_graph, jobs, chunksize=1)
    else:
        res = [_batched_graph(j) for j in jobs]
    ns = [r[0] for r in res]
    pre = [r[1] for r in res]
    rnds = [[r[2][k] for r in res] for k in range(rounds)]
    return ns, pre, rnds


def _oracle_batched_worker(work, warm, timed, barrier, queue):
    """One host process of the batched form's CPU baseline: its graphs' preload and
    warm-up rounds untimed, then the timed rounds between two barriers."""
    from oracle import oracle as O
    graphs = [(O.OraclePLDS(n), pre, rs) for n, pre, rs in work]
    for o, pre, rs in graphs:
        o.insert(pre)
        for ins, dele in rs[:warm]:
            o.insert(ins)
            o.delete(dele)
    barrier.wait()
    t0 = time.perf_counter()
    upd = 0
    for o, pre, rs in graphs:
        for ins, dele in rs[warm:warm + timed]:
            o.insert(ins)
            o.delete(dele)
            upd += ins.shape[0] + dele.shape[0]
    t1 = time.perf_counter()
    queue.put((upd, t0, t1))


def batched_cpu_baseline(ns, pre, rnds, warm: int, timed: int, every: int) -> dict:
    """The oracle as P independent processes (P = host cores) over a sample of the
    graphs (every `every`-th, split over the processes by the greedy size balance):
    the same preload and warm-up rounds untimed, then `timed` rounds; updates/s =
    the sampled updates over the wall time from the common start to the last end."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    sample = list(range(0, len(ns), every))
    procs_n = max(1, min(os.cpu_count() or 1, len(sample)))
    parts = shard_graphs([pre[i].shape[0] for i in sample], procs_n)
    barrier, queue = ctx.Barrier(procs_n), ctx.Queue()
    procs = []
    for part in parts:
        work = [(ns[sample[k]], pre[sample[k]], [rnds[r][sample[k]] for r in range(warm + timed)]) for k in part]
        p = ctx.Process(target=_oracle_batched_worker, args=(work, warm, timed, barrier, queue))
        p.start()
        procs.append(p)
    res = [queue.get() for _ in procs]
    for p in procs:
        p.join()
    upd = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": upd / wall, "unit": UNIT, "cores": procs_n, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"{len(sample)} of the {len(ns)} graphs (every {every}th), {timed} mixed rounds after the "
                      f"same preload and {warm} warm-up rounds, as {procs_n} independent oracle processes "
                      f"(graphs split by size); {upd} updates in {wall:.2f} s wall"}


def batched_results(P, ns, pre, rnds, warmup: int, tune_trials: int, plain_rounds: int,
                    autotune: bool = True, cpu_every: int = 16, cpu_rounds: int = 2, local: int = 0) -> dict:
    """The batched form on the given graphs (one launch per round of batches), the
    same rounds with the set's default knobs, the plain form looping over the graphs,
    and the oracle's CPU baseline."""
    import torch
    rounds = len(rnds)
    e0, o0 = P.PLDSSet.pack([(p_, np.zeros((0, 2), np.int32)) for p_ in pre])
    pre_dev = (torch.from_numpy(e0).cuda(), o0)
    packed = [P.PLDSSet.pack(r) for r in rnds]
    dev = [(torch.from_numpy(e).cuda(), o) for e, o in packed]
    upd = [int(o[-1]) for _, o in packed]
    w = min(warmup, rounds - 1)

    def timed_set(tuning, clk=None):
        """Preload, warm-up rounds, then the timed rounds; returns (seconds, set, per-round ms)."""
        S = P.PLDSSet(ns)
        if tuning:
            S.tune(**tuning)
        S.update(*pre_dev)
        for r in range(w):
            S.update(*dev[r])
        torch.cuda.synchronize()
        lat = []
        t0 = time.perf_counter()
        for r in range(w, rounds):
            t1 = time.perf_counter()
            S.update(*dev[r])
            lat.append(1e3 * (time.perf_counter() - t1))
        torch.cuda.synchronize()
        return time.perf_counter() - t0, S, lat

    tuning, t_tune = None, 0.0
    if autotune and w > 0:
        probe = P.PLDSSet(ns)
        t0 = time.perf_counter()
        tuning = probe.autotune([pre_dev] + dev[:w], timed_from=1, max_trials=tune_trials)
        t_tune = time.perf_counter() - t0
        probe.close()
    dt_default, S0, _ = timed_set(None)
    S0.close()
    with ClockSampler(local) as clk:
        dt, S, lat = timed_set(tuning)
    batched = sum(upd[w:]) / dt
    # the plain form: one synchronous insert and delete call per graph, graphs one after another
    G = [P.PLDS(n) for n in ns]
    for g, p_ in zip(G, pre):
        g.insert(torch.from_numpy(p_).cuda())
    for r in range(w):
        for g, (ins, dele) in zip(G, rnds[r]):
            g.insert(torch.from_numpy(ins).cuda())
            g.delete(torch.from_numpy(dele).cuda())
    nplain = min(rounds - w, plain_rounds)
    devr = [[(torch.from_numpy(i_).cuda(), torch.from_numpy(d_).cuda()) for i_, d_ in rnds[r]]
            for r in range(w, w + nplain)]
    torch.cuda.synchronize()
    plat = []
    t0 = time.perf_counter()
    for rr in devr:
        t1 = time.perf_counter()
        for g, (ins, dele) in zip(G, rr):
            g.insert(ins)
            g.delete(dele)
        plat.append(1e3 * (time.perf_counter() - t1))
    torch.cuda.synchronize()
    dtp = time.perf_counter() - t0
    plain = sum(upd[w:w + nplain]) / dtp
    same = all(np.array_equal(a.levels(), b.levels()) for a, b in zip(S.graphs, G)) if nplain == rounds - w else None
    S.close()
    for g in G:
        g.close()
    out = {"updates_per_s": batched, "rounds_timed": rounds - w, "warmup_rounds": w,
           "round_ms": {"mean": 1e3 * dt / (rounds - w), "p50": pct(lat, 50), "p99": pct(lat, 99),
                        "of": "host time of each round's call (submit to completion)"},
           "clocks": clk.summary(),
           "plain_loop": {"updates_per_s": plain, "rounds_timed": nplain,
                          "round_ms": {"mean": 1e3 * dtp / nplain, "p50": pct(plat, 50), "p99": pct(plat, 99)}},
           "speedup_vs_plain": batched / plain, "levels_equal_plain": same,
           "autotune": {"knobs": tuning, "seconds": t_tune, "trials_max": tune_trials,
                        "sample": "preload + warm-up rounds (untimed)",
                        "default_knobs_updates_per_s": sum(upd[w:]) / dt_default},
           "workload": {"graphs": len(ns), "total_vertices": int(sum(ns)),
                        "updates_per_round": int(np.mean(upd))}}
    if cpu_every:
        out["cpu_baseline"] = batched_cpu_baseline(ns, pre, rnds, w, min(cpu_rounds, rounds - w), cpu_every)
    return out


def device_checks(P, g, n, present, tables):
    """Counters by definition and Invariants 1-2 computed on the device with torch
    (graphs too large for the host check): deg, up (neighbours on the same level or
    above) and up* (on the level below or above) recounted from the edge list and
    the levels, compared with the structure's own counters."""
    import torch
    dev = present.device
    lv = torch.empty(n, dtype=torch.int32, device=dev)
    g.levels(lv)
    mine = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(3)]
    g.counters(mine)
    torch.cuda.synchronize()
    lv = lv.long()
    deg, up, ups = (torch.zeros(n, dtype=torch.int64, device=dev) for _ in range(3))
    chunk = 1 << 26
    for s0 in range(0, present.shape[0], chunk):
        u = present[s0:s0 + chunk, 0].long()
        v = present[s0:s0 + chunk, 1].long()
        lu, lw = lv[u], lv[v]
        one = torch.ones_like(u)
        deg.index_add_(0, u, one)
        deg.index_add_(0, v, one)
        up.index_add_(0, u, (lw >= lu).long())
        up.index_add_(0, v, (lu >= lw).long())
        ups.index_add_(0, u, (lw >= lu - 1).long())
        ups.index_add_(0, v, (lu >= lw - 1).long())
    upmax = torch.as_tensor(np.asarray(tables[0], np.int64), device=dev)
    dnmin = torch.as_tensor(np.asarray(tables[1], np.int64), device=dev)
    Lg = g.Lg
    pos = lv > 0
    return {"deg_by_definition": bool(torch.equal(deg, mine[0].long())),
            "up_by_definition": bool(torch.equal(up, mine[1].long())),
            "upstar_by_definition": bool(torch.equal(ups, mine[2].long())),
            "invariant1": bool((up <= upmax[lv // Lg]).all()),
            "invariant2": bool((ups[pos] >= dnmin[(lv[pos] - 1) // Lg]).all())}


def unique_edges_device(pairs):
    """Distinct non-loop edges of a device pair list, canonical (u < v), int32 [k, 2]."""
    import torch
    keys = []
    for s0 in range(0, pairs.shape[0], 1 << 27):
        u = pairs[s0:s0 + (1 << 27), 0].long()
        v = pairs[s0:s0 + (1 << 27), 1].long()
        keep = u != v
        u, v = u[keep], v[keep]
        keys.append(torch.minimum(u, v) * (1 << 32) + torch.maximum(u, v))
    k = torch.unique(torch.cat(keys))
    del keys
    return torch.stack([(k >> 32).int(), (k & 0xFFFFFFFF).int()], 1).contiguous()


def large_parity(P, gen, n, B, nb, gold_path):
    """The first nb batches of the large insertion stream on a fresh handle, each
    batch's level and counter digests against the oracle's (written by
    tests/golden/make_large_digests.py from oracle/ only).  Untimed."""
    import torch
    if not gold_path.exists():
        return {"checked": 0, "note": f"{gold_path.name} not present"}
    gold = json.loads(gold_path.read_text())
    recs = gold.get("ins", [])[:nb]
    if gold["n"] != n or gold["batch"] != B or gold["perm_sha256"] != sha_i32(gen.perm):
        return {"checked": 0, "note": "the golden file describes another stream"}
    g = P.PLDS(n)
    ok_lv = ok_ct = ok_n = True
    for j, r in enumerate(recs):
        b = gen.draws_torch(r["start"], r["size"])
        g.insert(b)
        st = g.stats()
        d, u, s_ = g.counters()
        ok_lv &= sha_i32(g.levels()) == r["levels"]
        ok_ct &= sha_i32(d, u, s_) == r["counters"]
        ok_n &= all(st[k] == r[k] for k in ("valid", "rounds", "moves", "visits"))
        del b
    g.close()
    torch.cuda.empty_cache()
    return {"checked": len(recs), "updates": sum(r["size"] for r in recs), "levels_equal": bool(ok_lv),
            "counters_equal": bool(ok_ct), "work_counts_equal": bool(ok_n),
            "against": "oracle digests after every batch (" + gold_path.name + ")"}


def sha_i32(*arrays) -> str:
    h = hashlib.sha256()
    for x in arrays:
        h.update(np.ascontiguousarray(x, dtype="<i4").tobytes())
    return h.hexdigest()


def run_large(args):
    """The large configuration: a Chung-Lu graph shaped like a billion-edge social
    graph (n = 41.7M, 1.2B drawn pairs, exponent 2.1; counter-based draws made on the
    device) and a 24M-vertex road-like grid, plain form, device-resident inputs; Ins /
    Mix / Del protocols at batches of 1e7 and 1e6, device-side property checks on the
    loaded graph, and the first 10^8 insertions checked against the oracle's digests."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    torch.cuda.set_device(0)
    n, m = args.large_n, args.large_m
    B7, B6 = 10_000_000, 1_000_000
    t0 = time.perf_counter()
    gen = W.ChungLuDraws(n, m, 2.1, seed=1)
    raw = gen.draws_torch(0, m)  # the insertion stream: raw pairs in draw order
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    parity = large_parity(P, gen, n, B7, 10, ROOT / "tests" / "golden" / "chunglu41m_first1e8_digests.json")

    def timed(calls):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(calls) + 1)]
        upd = 0
        torch.cuda.synchronize()
        evs[0].record()
        for i, (fn, b) in enumerate(calls):
            fn(b)
            upd += b.shape[0]
            evs[i + 1].record()
        torch.cuda.synchronize()
        lat = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(calls))]
        return {"updates_per_s": upd / (evs[0].elapsed_time(evs[-1]) / 1e3), "batches": len(calls),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}

    out = {}
    g = P.PLDS(n)
    k = int(0.9 * m)
    # build: the first 90 % of the draws in batches of 1e7 (the Ins protocol at 1e7)
    out["ins_1e7"] = timed([(g.insert, raw[s:min(s + B7, k)]) for s in range(0, k, B7)])
    st = g.stats()
    present = unique_edges_device(raw[:k])
    out["loaded"] = {"draws": k, "edges": int(present.shape[0]), "device_bytes": st["device_bytes"],
                     "pool_slots": st["pool_slots_cap"]}
    out["checks_loaded"] = device_checks(P, g, n, present, g.tables())
    # Mix on the 90 %-loaded graph: insert edges of the last 10 % of the draws that are
    # not present yet, delete from a shuffled present pool
    later = unique_edges_device(raw[k:])
    del raw
    pk = present[:, 0].long() * (1 << 32) + present[:, 1].long()
    lk = later[:, 0].long() * (1 << 32) + later[:, 1].long()
    pos = torch.searchsorted(pk, lk).clamp_(max=pk.numel() - 1)
    absent = W.shuffled_device(later[pk[pos] != lk], 13)
    del pk, lk, pos, later
    present = W.shuffled_device(present, 12)
    ai, pi = 0, 0

    def mixed(B, count):
        nonlocal ai, pi
        calls = []
        for _ in range(count):
            h = B // 2
            calls.append((g.insert, absent[ai:ai + h]))
            calls.append((g.delete, present[pi:pi + h]))
            ai += h
            pi += h
        return calls

    out["mix_1e7"] = timed(mixed(B7, 3))
    out["mix_1e6"] = timed(mixed(B6, 10))
    out["ins_1e6"] = timed([(g.insert, absent[ai + j * B6:ai + (j + 1) * B6]) for j in range(5)])
    ai += 5 * B6
    out["del_1e6"] = timed([(g.delete, present[pi + j * B6:pi + (j + 1) * B6]) for j in range(5)])
    pi += 5 * B6
    # Del at 1e7: everything still present
    rest = torch.cat([present[pi:], absent[:ai]])
    out["del_1e7"] = timed([(g.delete, rest[s:s + B7]) for s in range(0, rest.shape[0], B7)])
    out["empty_after_del"] = bool(int(g.levels().max()) == 0 and int(g.counters()[0].max()) == 0)
    g.close()
    del present, absent, rest
    torch.cuda.empty_cache()
    # the road-like contrast: 24M-vertex grid, degree <= 4 plus 10 % diagonals
    side = args.grid_side
    ge = torch.from_numpy(W.shuffled(W.grid2d(side, 0.1, seed=1), 13)).cuda()
    ng = side * side
    g = P.PLDS(ng)
    grid = {"n": ng, "m": int(ge.shape[0])}
    grid["ins_1e7"] = timed([(g.insert, ge[s:s + B7]) for s in range(0, ge.shape[0], B7)])
    grid["checks_loaded"] = device_checks(P, g, ng, ge, g.tables())
    grid["max_level"] = int(g.levels().max())
    gd = W.shuffled_device(ge, 14)
    grid["del_1e7"] = timed([(g.delete, gd[s:s + B7]) for s in range(0, gd.shape[0], B7)])
    g.close()
    line = {"metric": "edge updates/s, large graphs (plain form)", "value": out["ins_1e7"]["updates_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": out["ins_1e7"]["batches"], "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic", "form": "large",
            "config": {"workload": f"Chung-Lu n={n}, {m} drawn pairs, exponent 2.1 (counter-based draws "
                                   f"made on the device, {t_gen:.1f} s); grid {side}x{side} with 10% diagonals",
                       "value_is": "Ins protocol at batch 1e7 while loading 90% of the draws (raw pairs: "
                                   "repeats and self-loops included, dropped by the batch rules)"},
            "parity_first_1e8": parity, "chung_lu": out, "grid": grid}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """--form batched: one JSON line.  Under torchrun (N > 1 ranks) every rank takes
    its share of the graphs by the greedy size balance and runs them as its own set;
    value = the updates of all ranks over the slowest rank's time (no data-path
    collective: the graphs are independent)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    ns, pre, rnds = make_batched(args.graphs, args.rounds)
    mine = shard_graphs([p_.shape[0] for p_ in pre], world)[rank]
    ns_r = [ns[i] for i in mine]
    pre_r = [pre[i] for i in mine]
    rnds_r = [[r[i] for i in mine] for r in rnds]
    res = batched_results(P, ns_r, pre_r, rnds_r, args.warmup, args.tune_trials, args.plain_rounds,
                          autotune=not args.no_autotune, cpu_every=4 if world == 1 else 0, cpu_rounds=args.rounds,
                          local=local)
    w = res["warmup_rounds"]
    upd = sum(sum(i.shape[0] + d.shape[0] for i, d in rnds_r[r]) for r in range(w, args.rounds))
    secs = upd / res["updates_per_s"]
    if dist:
        dist.barrier()
    upd_all, secs_max = whole_job(dist, upd, secs, "cuda")
    if rank == 0:
        line = {"metric": "edge updates/s, batched form (one launch per round of batches)",
                "value": upd_all / secs_max, "unit": UNIT, "n_gpus": world, "steps": args.rounds - w,
                "warmup": w, "ms_per_step": 1e3 * secs_max / (args.rounds - w), "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "form": "batched",
                "config": {"workload": f"{args.graphs} Chung-Lu graphs, n log-uniform [1e3,1e5], exponent "
                                       f"U[2.1,2.8], avg degree U[4,32], half preloaded, {args.rounds} mixed rounds "
                                       "of 1-10% of edges",
                           "parallelism": f"graphs split over {world} ranks by size (greedy)"},
                "rank0": res}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def make_serving_stream(e: np.ndarray, requests: int, seed: int = 5):
    """Open-loop request stream on a graph preloaded with 90 % of its edges: sizes
    log-uniform in [10, 1e6], insertion or deletion with equal probability
    (insertions from the absent pool, deletions from the present pool, both queues),
    and a full coreness query after every 20 update batches."""
    rng = np.random.default_rng(seed)
    e = e[rng.permutation(e.shape[0])]
    k = int(0.9 * e.shape[0])
    pre, present, absent = e[:k], e[:k].copy(), e[k:].copy()
    reqs, nb = [], 0
    while len(reqs) < requests:
        if nb and nb % 20 == 0 and (not reqs or reqs[-1][0] != 2):
            reqs.append((2, None))
            continue
        size = int(np.exp(rng.uniform(np.log(10), np.log(1e6))))
        if rng.random() < 0.5:
            size = min(size, absent.shape[0])
            b, absent = absent[:size], absent[size:]
            present = np.concatenate([present, b])
            reqs.append((0, np.ascontiguousarray(b)))
        else:
            j = rng.integers(0, max(1, present.shape[0] - size))
            b = present[j:j + size]
            present = np.concatenate([present[:j], present[j + size:]])
            absent = np.concatenate([absent, b])
            reqs.append((1, np.ascontiguousarray(b)))
        nb += 1
    return np.ascontiguousarray(pre), reqs


def serving_cpu_baseline(n: int, reqs, budget: int = 1_000_000, min_requests: int = 40) -> dict:
    """The oracle (1 core) on the stream's first requests (at least `min_requests`,
    until `budget` updates), applied to an empty graph of the same n (building the
    preloaded 90 % state would take the oracle over ten minutes)."""
    from oracle import oracle as O
    o = O.OraclePLDS(n)
    upd, k = 0, 0
    t0 = time.perf_counter()
    for op, b in reqs:
        if op == 2:
            o.coreness()
        elif op == 0:
            o.insert(b)
        else:
            o.delete(b)
        k += 1
        upd += 0 if b is None else b.shape[0]
        if upd >= budget and k >= min_requests:
            break
    dt = time.perf_counter() - t0
    return {"value": upd / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu": host_cpu(),
            "sample": f"the first {k} requests ({upd} updates) of the same request stream applied to an empty "
                      f"{n}-vertex graph by the sequential oracle, {dt:.1f} s on 1 host core"}


def serving_results(P, n: int, m: int, requests: int, slots: int, local: int = 0, cpu: bool = True) -> dict:
    """The serving form against the plain form on the same open-loop stream:
    capacities with the whole stream submitted at once, then p50/p99 latency (from a
    request's scheduled arrival to the host seeing it done) at 70 % and 90 % of the
    plain form's capacity; estimates of the merged and the unmerged loops compared
    per vertex on the final graph (the same edges, different batch boundaries)."""
    import torch
    e = W.chung_lu(n, m, 2.2, seed=1)
    pre, reqs = make_serving_stream(e, requests)
    pre_d = torch.from_numpy(pre).cuda()
    pinned = [(op, torch.from_numpy(b).pin_memory() if b is not None else None) for op, b in reqs]
    qout = torch.empty(n, dtype=torch.float64).pin_memory()
    upd_total = sum(b.shape[0] for op, b in reqs if b is not None)

    def preloaded():
        g = P.PLDS(n)
        for s0 in range(0, pre_d.shape[0], 1_000_000):
            g.insert(pre_d[s0:s0 + 1_000_000])
        torch.cuda.synchronize()
        return g

    def plain_call(g, op, b):
        if op == 2:
            g.coreness(qout.numpy())
        elif op == 0:
            g.insert(b)
        else:
            g.delete(b)

    # capacity of the plain form: the stream back to back
    g = preloaded()
    t0 = time.perf_counter()
    for op, b in pinned:
        plain_call(g, op, b)
    cap_s = time.perf_counter() - t0
    g.close()
    results = {"plain_capacity_updates_per_s": upd_total / cap_s, "stream_seconds_back_to_back": cap_s}

    # capacity of the served forms: the whole stream submitted at once
    final = {}
    for form, merge in (("served", -1), ("served_unmerged", 0)):
        g = preloaded()
        sv = P.Server(g, slots=slots, max_batch=2_000_000, merge_max_edges=merge)
        t0 = time.monotonic_ns()
        for op, b in pinned:
            if op == 2:
                sv.submit(2, out=qout.numpy())
            else:
                sv.submit(op, edges=b)
        sv.drain()
        done = sv.poll(4096)
        sv.close()
        final[form] = g.coreness()
        g.close()
        span = (max(r["done_ns"] for r in done) - t0) * 1e-9
        results[f"{form}_capacity_updates_per_s"] = upd_total / span
        results[f"{form}_device_batches_back_to_back"] = sum(r["batch_first"] == r["ticket"] for r in done)
    a, b = final["served"], final["served_unmerged"]
    nz = (a > 0) & (b > 0)
    ratio = np.maximum(a[nz] / b[nz], b[nz] / a[nz])
    results["merged_vs_unmerged_estimates"] = {
        "max_ratio": float(ratio.max()) if ratio.size else 1.0, "mean_ratio": float(ratio.mean()) if ratio.size else 1.0,
        "zero_mismatch": int(((a > 0) != (b > 0)).sum()),
        "of": "per-vertex coreness estimates after the whole stream, continuous batching vs one batch per request"}

    clocks = {}
    for load in (0.7, 0.9):
        rate = load * len(reqs) / cap_s
        rng = np.random.default_rng(99)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        for form in ("plain", "served", "served_unmerged"):
            g = preloaded()
            lat = np.zeros(len(reqs))
            sizes = []
            with ClockSampler(local) as clk:
                if form == "plain":
                    t0 = time.monotonic_ns()
                    for i, (op, b) in enumerate(pinned):
                        due = t0 + int(arrivals[i] * 1e9)
                        while time.monotonic_ns() < due:
                            pass
                        plain_call(g, op, b)
                        lat[i] = (time.monotonic_ns() - due) * 1e-9
                    span = (time.monotonic_ns() - t0) * 1e-9
                else:
                    sv = P.Server(g, slots=slots, max_batch=2_000_000, merge_max_edges=-1 if form == "served" else 0)
                    done = {}
                    t0 = time.monotonic_ns()
                    for i, (op, b) in enumerate(pinned):
                        due = t0 + int(arrivals[i] * 1e9)
                        while time.monotonic_ns() < due:
                            for r in sv.poll():
                                done[r["ticket"]] = r
                        if op == 2:
                            sv.submit(2, out=qout.numpy())
                        else:
                            sv.submit(op, edges=b)
                    while len(done) < len(reqs):
                        for r in sv.poll():
                            done[r["ticket"]] = r
                    span = (max(r["done_ns"] for r in done.values()) - t0) * 1e-9
                    for i in range(len(reqs)):
                        lat[i] = (done[i]["done_ns"] - (t0 + int(arrivals[i] * 1e9))) * 1e-9
                    sizes = [r["batch_size"] for r in done.values() if r["batch_first"] == r["ticket"]]
                    sv.close()
            g.close()
            clocks[f"{form}@{int(load * 100)}%"] = clk.summary()
            results[f"{form}@{int(load * 100)}%"] = {
                "p50_ms": pct(lat * 1e3, 50), "p99_ms": pct(lat * 1e3, 99), "mean_ms": float(lat.mean() * 1e3),
                "updates_per_s": upd_total / span, "makespan_s": span,
                **({"device_batches": len(sizes), "max_requests_per_batch": int(max(sizes))} if sizes else {})}
    out = {"capacity_updates_per_s": results["served_capacity_updates_per_s"],
           "p50_ms_at_90pct": results["served@90%"]["p50_ms"], "p99_ms_at_90pct": results["served@90%"]["p99_ms"],
           "plain": {"capacity_updates_per_s": results["plain_capacity_updates_per_s"],
                     "p50_ms_at_90pct": results["plain@90%"]["p50_ms"],
                     "p99_ms_at_90pct": results["plain@90%"]["p99_ms"]},
           "workload": {"graph": f"Chung-Lu n={n}, m={e.shape[0]}, exponent 2.2, 90% preloaded",
                        "requests": len(reqs), "updates": upd_total, "slots": slots,
                        "stream": "sizes log-uniform [10,1e6], 50/50 Ins/Del, coreness query every 20 batches, "
                                  "Poisson arrivals at 70% and 90% of the plain form's capacity, inputs in "
                                  "pinned host memory",
                        "forms": "served = continuous batching (merged runs of waiting requests, logged "
                                 "schedule); served_unmerged = the same loop, one batch per request"},
           "results": results, "clocks": clocks}
    if cpu:
        out["cpu_baseline"] = serving_cpu_baseline(n, reqs)
    return out


def run_serving(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    torch.cuda.set_device(0)
    res = serving_results(P, args.serve_n, args.serve_m, args.requests, args.slots)
    line = {"metric": "edge updates/s and p50/p99 batch latency, serving form (device-resident request loop)",
            "value": res["capacity_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": res["workload"]["requests"],
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "form": "serving", "config": {"workload": res["workload"]["graph"]}, **res}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=29)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--batch", type=int, default=1_000_000)
    ap.add_argument("--ref-batch", type=int, default=100_000)
    ap.add_argument("--cpu-batch", type=int, default=500_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-protocols", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="leave the serving and batched forms out of the line")
    ap.add_argument("--dump-recs", default=None, help="write per-step kernel records (JSON) to this path")
    ap.add_argument("--form", default="plain", choices=["plain", "batched", "serving", "large"])
    ap.add_argument("--large-n", type=int, default=41_700_000)
    ap.add_argument("--large-m", type=int, default=1_200_000_000)
    ap.add_argument("--grid-side", type=int, default=4899)
    ap.add_argument("--serve-n", type=int, default=4_800_000)
    ap.add_argument("--serve-m", type=int, default=43_000_000)
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--slots", type=int, default=32)
    ap.add_argument("--graphs", type=int, default=512)
    ap.add_argument("--rounds", type=int, default=20)
    ap.add_argument("--plain-rounds", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-trials", type=int, default=16)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.form == "batched":
        return run_batched(args)
    if args.form == "serving":
        return run_serving(args)
    if args.form == "large":
        return run_large(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P

    e, ins_h, del_h, steps = make_stream(args.scale, args.batch)
    n = 1 << args.scale
    ins_d = torch.from_numpy(ins_h).cuda()
    del_d = torch.from_numpy(del_h).cuda()
    core_d = torch.empty(n, dtype=torch.float64, device="cuda")

    def run_steps(g, k0, count, host=False, pinned=None, core_h=None, lat=None):
        upd, recs = 0, []
        for k in range(k0, k0 + count):
            kind, a, b = steps[k % len(steps)]
            if host:
                src = pinned[kind][a:b]
            else:
                src = (ins_d if kind == "ins" else del_d)[a:b]
            t1 = time.perf_counter()
            (g.insert if kind == "ins" else g.delete)(src)  # synchronous: returns when the batch is done
            if lat is not None:
                lat.append(1e3 * (time.perf_counter() - t1))
            recs.append((kind, g.stats()))
            g.coreness(core_h if host else core_d)
            upd += b - a
        return upd, recs

    g = P.PLDS(n)
    run_steps(g, 0, args.warmup)
    launches0 = g.stats()["launches"]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    host_lat = []
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")  # lets an ncu capture select the timed steps' kernels
        ev0.record()
        upd, recs = run_steps(g, args.warmup, args.steps, lat=host_lat)
        ev1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = g.stats()["launches"] - launches0
    g.close()
    upd_all, t_max_s = whole_job(dist, upd, ms / 1e3, "cuda")
    valid_all, _ = whole_job(dist, sum(r["valid"] for _, r in recs), ms / 1e3, "cuda")
    t_max = t_max_s * 1e3
    value = upd_all / t_max_s

    # roofline: algorithmic bytes of the executed work / event-timed duration, for the
    # level-rounds kernel (the dominant one) and for the whole launch sequence of a batch
    # (step kernels + rounds kernel); both measured on the handle's stream
    nb = len(recs)
    kern_ns = sum(r["kernel_ns"] for _, r in recs)
    pre_ns = sum(r["pre_ns"] for _, r in recs)
    rnd_ns = kern_ns - pre_ns
    abytes = sum(algo_bytes(r, kind) for kind, r in recs)
    pbytes = sum(algo_bytes_steps(r) for _, r in recs)
    sbytes = sum(algo_bytes_degree(r) for _, r in recs)
    xbytes = sum(algo_bytes_with_skipped(r, kind) for kind, r in recs)
    peak, peak_src = measured_peaks()

    def gbs(b, ns):
        return b / (ns / 1e9) / 1e9 if ns > 0 else None

    def frac(a):
        return a / peak if a else None

    cur = NCU_TRAFFIC["kernel_sha"] == kernel_sha()
    r_traffic = (NCU_TRAFFIC["rounds_dram_per_algo_byte"] * (abytes - pbytes) / nb
                 if cur and NCU_TRAFFIC["rounds_dram_per_algo_byte"] else None)
    b_traffic = (NCU_TRAFFIC["batch_dram_per_algo_byte"] * abytes / nb
                 if cur and NCU_TRAFFIC["batch_dram_per_algo_byte"] else None)
    if args.dump_recs:  # per timed step: algorithmic bytes and durations (matches ncu launch lists)
        with open(args.dump_recs, "w") as f:
            json.dump([{"kind": kind, "algo_bytes": algo_bytes(r, kind), "algo_bytes_steps": algo_bytes_steps(r),
                        "algo_bytes_degree": algo_bytes_degree(r), "kernel_ns": r["kernel_ns"],
                        "pre_ns": r["pre_ns"], "launches": r["launches"], "valid": r["valid"]}
                       for kind, r in recs], f)
    a_rnd = gbs(abytes - pbytes, rnd_ns)
    s_rnd = gbs(sbytes - pbytes, rnd_ns)
    a_seq = gbs(abytes, kern_ns)
    s_seq = gbs(sbytes, kern_ns)
    a_pre = gbs(pbytes, pre_ns)
    roof = {"bound": "hbm", "achieved": a_rnd, "peak": peak, "unit": "GB/s", "frac": frac(a_rnd),
            "traffic": r_traffic, "kernel": "k_batch_grid", "peak_source": peak_src,
            "kernel_ms_per_launch": rnd_ns / 1e6 / nb,
            "algo_bytes_per_launch": (abytes - pbytes) / nb,
            "definition": "executed work of the level rounds: 4 B per level change, 8 B per neighbour "
                          "examined (insertion moves: up-neighbours; deletion moves: all), 8 B per neighbour "
                          "read by a desire-level evaluation; skipped pure rounds left out",
            "degree_definition": {"algo_bytes_per_launch": (sbytes - pbytes) / nb, "achieved": s_rnd,
                                  "frac": frac(s_rnd),
                                  "definition": "executed work, every move at its degree + 8 B per affected "
                                                "neighbour"},
            "batch_sequence": {"kernels": "step kernels (8 per insertion batch, 6 per deletion batch) "
                                          "+ k_batch_grid, one batch call",
                               "ms_per_batch": kern_ns / 1e6 / nb, "algo_bytes_per_batch": abytes / nb,
                               "achieved": a_seq, "frac": frac(a_seq), "traffic": b_traffic,
                               "degree_algo_bytes_per_batch": sbytes / nb, "degree_achieved": s_seq,
                               "degree_frac": frac(s_seq)},
            "step_kernels": {"ms_per_batch": pre_ns / 1e6 / nb, "algo_bytes_per_batch": pbytes / nb,
                             "achieved": a_pre, "frac": frac(a_pre),
                             "definition": "8 B per submitted edge + 64 B per applied update"},
            "with_skipped_rounds": {"algo_bytes_per_batch": xbytes / nb,
                                    "note": "the skipped pure rounds counted as Algorithm 2 would run them; "
                                            "not a bandwidth figure"}}

    # e2e: the same steps through the C ABI with pinned host buffers (H2D of the batch
    # and D2H of every vertex's coreness inside the timed region), fresh graph
    e2e = None
    if not args.no_e2e:
        pinned = {"ins": torch.from_numpy(ins_h).pin_memory().numpy(),
                  "del": torch.from_numpy(del_h).pin_memory().numpy()}
        core_h = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        g2 = P.PLDS(n)
        run_steps(g2, 0, args.warmup, host=True, pinned=pinned, core_h=core_h)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        upd2, _ = run_steps(g2, args.warmup, args.steps, host=True, pinned=pinned, core_h=core_h)
        torch.cuda.synchronize()
        dt2 = time.perf_counter() - t0
        g2.close()
        upd2_all, dt2 = whole_job(dist, upd2, dt2, "cuda")
        e2e = {"value": upd2_all / dt2, "unit": UNIT, "h2d_bytes_per_step": 8 * upd2 / args.steps,
               "d2h_bytes_per_step": 8 * n}

    lat_ms = [r["kernel_ns"] / 1e6 for _, r in recs]
    protocols = None
    forms = None
    if world == 1 and not args.no_protocols:
        protocols = run_protocols(P, n, e, ins_d, del_d)
        # the paper's optimised variant: ceil(log_{1+delta} m / 50) levels per group
        lg_opt = P.opt_levels_per_group(int(e.shape[0]))
        protocols["plds_opt"] = {"levels_per_group": lg_opt,
                                 **run_protocols(P, n, e, ins_d, del_d, levels_per_group=lg_opt,
                                                 sizes=(1_000_000,))}
        # the experiments' filter+sort insertion variant (same levels, its own rounds)
        protocols["jump"] = run_protocols(P, n, e, ins_d, del_d, jump=True)
    if world == 1 and not args.no_forms:
        del ins_d, del_d
        torch.cuda.empty_cache()
        forms = {"serving": serving_results(P, args.serve_n, args.serve_m, args.requests, args.slots, local,
                                            cpu=not args.no_cpu_baseline)}
        ns_b, pre_b, rnds_b = make_batched(args.graphs, args.rounds)
        forms["batched"] = batched_results(P, ns_b, pre_b, rnds_b, 3, min(args.tune_trials, 8), args.plain_rounds,
                                           cpu_every=0 if args.no_cpu_baseline else 4, cpu_rounds=args.rounds,
                                           local=local)

    phases = {}
    for kind in ("ins", "del"):
        sel = [(r, steps[(args.warmup + i) % len(steps)]) for i, (_, r) in enumerate(recs)
               if steps[(args.warmup + i) % len(steps)][0] == kind]
        if sel:
            ns = sum(r["kernel_ns"] for r, _ in sel)
            phases[kind] = {"steps": len(sel), "updates_per_s_kernel": sum(s[2] - s[1] for _, s in sel) / (ns / 1e9),
                            "rounds_counted": sum(r["rounds"] for r, _ in sel),
                            "rounds_run": sum(r["rounds"] - r["skipped_rounds"] for r, _ in sel)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample(args.scale, ins_h, args.cpu_batch)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": plain_config(args, n, int(e.shape[0]), world),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "valid_updates_per_s": valid_all / t_max_s,
        "phases": phases,
        "batch_latency_ms": {"kernel": {"p50": pct(lat_ms, 50), "p99": pct(lat_ms, 99)},
                             "submit_to_completion": {"p50": pct(host_lat, 50), "p99": pct(host_lat, 99)},
                             "of": "each timed step's batch call: its kernel (CUDA events), and the host time "
                                   "from the call to its return (the call is synchronous)"},
        "protocols": protocols,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
