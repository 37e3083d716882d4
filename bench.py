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

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 (under torchrun) runs N independent replicas (a single graph's level
rounds do not shard); value = all ranks' updates / max time.
--impl reference times the sequential CPU oracle on the host cores on bounded
samples of the same stream.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
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

# dram bytes / algorithmic bytes of the batch kernel, from the ncu capture
# summarised in profiles/ (kernel source hash at capture time); traffic is
# reported as null when the kernel source has changed since.
NCU_TRAFFIC = {"kernel_sha": "b311bada918cc187", "dram_per_algo_byte": 0.2269,
               "capture": "ncu DRAM counters of every k_batch_grid launch of the R-MAT 20 Ins and Del protocols"}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in sorted((ROOT / "paper_2106_03824_gb300" / "csrc").iterdir()):
        if f.suffix in (".cu", ".cuh", ".h", ".cpp"):
            h.update(f.read_bytes())
    return h.hexdigest()[:16]


def whole_job(dist, updates: float, seconds: float, device: str):
    """The whole-job figures of a replicas run: the updates of every rank and the
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


def algo_bytes(s: dict) -> int:
    """Algorithmic bytes of one batch kernel launch: 8 B per submitted edge; 64 B per
    applied update (2 probes + 2 slot writes of 4 B, 6 counter read-modify-writes of
    8 B); 4 B per level change; 8 B (id + level) per neighbour a move must examine --
    an insertion move its up-neighbours (up_visits), a deletion move all its
    neighbours (visits); 8 B per neighbour read by a desire-level evaluation."""
    moved = s["up_visits"] if s.get("up_visits") else s["visits"]
    return 8 * s["submitted"] + 64 * s["valid"] + 4 * s["moves"] + 8 * moved + 8 * s["dl_visits"]


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


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


def make_stream(scale: int, batch: int, seed: int = 1):
    e = W.rmat(scale, 16, seed=seed)
    ins = W.shuffled(e, 11)
    dele = W.shuffled(e, 12)
    steps = [("ins", s, min(s + batch, e.shape[0])) for s in range(0, e.shape[0], batch)]
    steps += [("del", s, min(s + batch, e.shape[0])) for s in range(0, e.shape[0], batch)]
    return e, ins, dele, steps


def run_protocols(P, n, e, ins_d, del_d, mix_batches=10, seed=3, levels_per_group=0,
                  sizes=(1_000_000, 100_000)):
    """The experiments' Ins / Del / Mix protocols on the same graph, plain form,
    device-resident inputs: Ins all edges from empty and Del them all, in batches of
    1e6 and 1e5; Mix = 50/50 insert/delete batches of 1e6 on a 90 %-loaded graph
    (untimed preload).  Per protocol: updates/s over the whole sequence and the
    p50/p99 of the per-batch latency, both from CUDA events on the handle's stream."""
    import torch

    def timed(g, calls):
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
        tot = evs[0].elapsed_time(evs[-1])
        return {"updates_per_s": upd / (tot / 1e3), "batches": len(calls),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}

    out = {}
    for B in sizes:
        tag = "1e6" if B == 1_000_000 else "1e5"
        g = P.PLDS(n, levels_per_group=levels_per_group)
        out[f"ins_{tag}"] = timed(g, [(g.insert, ins_d[s:s + B]) for s in range(0, ins_d.shape[0], B)])
        if B == sizes[0] and levels_per_group == 0:
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
    g = P.PLDS(n, levels_per_group=levels_per_group)
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
    return {"value": b.shape[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {b.shape[0]} edges of the first Ins batch of the same R-MAT scale-{scale} "
                      f"stream, applied as one batch to the empty graph ({dt:.1f} s on 1 host core; the "
                      f"full 10^6-edge batch takes minutes)"}


def plain_config(args, n: int, m: int, world: int) -> dict:
    """The workload of the default (plain-form) bench line; the reference arm reports the same."""
    return {"workload": f"rmat{args.scale}_ef16_B{args.batch:.0e}_ins_del_cycle".replace("+0", ""),
            "graph": f"R-MAT scale {args.scale}, (.57,.19,.19,.05), edge factor 16, symmetrised, deduplicated",
            "n": n, "m": m, "batch": args.batch, "delta": 0.4, "lambda": 3,
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
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": plain_config(args, 1 << args.scale, int(e.shape[0]), int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the sequential CPU oracle as it stands, on 1 host core: {args.steps} "
                                       f"consecutive Ins batches of {b} edges of the same stream from the empty "
                                       f"graph, after {args.warmup} warm-up batches (a full {args.batch}-edge "
                                       f"batch takes the oracle minutes)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def make_batched(graphs: int, rounds: int, seed: int = 7):
    """graphs Chung-Lu graphs (n log-uniform in [1e3,1e5], exponent U[2.1,2.8], average
    degree U[4,32]); half of each graph's edges preloaded (shuffled), then `rounds`
    mixed batches per graph, each inserting 0.5-5 % of its edges taken from the
    absent pool and deleting as many present ones (1-10 % of its edges in total);
    pools are queues, so a deleted edge can come back in a later round."""
    rng = np.random.default_rng(seed)
    ns, pre, rnds = [], [], [[] for _ in range(rounds)]
    for i in range(graphs):
        n = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
        e = W.chung_lu(n, int(n * rng.uniform(4, 32) / 2), rng.uniform(2.1, 2.8), seed=seed * 100003 + i)
        e = e[rng.permutation(e.shape[0])]
        half = e.shape[0] // 2
        ns.append(n)
        pre.append(np.ascontiguousarray(e[:half]))
        present, absent = e[:half], e[half:]
        for r in range(rounds):
            k = max(1, int(rng.uniform(0.005, 0.05) * e.shape[0]))
            k = min(k, present.shape[0], absent.shape[0])
            ins, dele = absent[:k], present[:k]
            rnds[r].append((np.ascontiguousarray(ins), np.ascontiguousarray(dele)))
            absent = np.concatenate([absent[k:], dele])
            present = np.concatenate([present[k:], ins])
    return ns, pre, rnds


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


def run_large(args):
    """The large configuration: a Chung-Lu graph shaped like a billion-edge social
    graph (n = 41.7M, ~1.2B edges, exponent 2.1) and a 24M-vertex road-like grid,
    plain form, device-resident inputs; Ins / Mix / Del protocols at batches of 1e7
    and 1e6, device-side property checks on the loaded graph."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    torch.cuda.set_device(0)
    n, m = args.large_n, args.large_m
    t0 = time.perf_counter()
    e = W.shuffled_device(W.chung_lu_device(n, m, 2.1, seed=1), 11)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    m = int(e.shape[0])

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
    B7, B6 = 10_000_000, 1_000_000
    # build: the first 90 % in batches of 1e7 (the Ins protocol at 1e7)
    out["ins_1e7"] = timed([(g.insert, e[s:min(s + B7, k)]) for s in range(0, k, B7)])
    st = g.stats()
    out["loaded"] = {"edges": k, "device_bytes": st["device_bytes"], "pool_slots": st["pool_slots_cap"]}
    out["checks_loaded"] = device_checks(P, g, n, e[:k], g.tables())
    # Mix on the 90 %-loaded graph: insert from the absent 10 %, delete from a shuffled present pool
    present = W.shuffled_device(e[:k], 12)
    ai, pi = k, 0

    def mixed(B, count):
        nonlocal ai, pi
        calls = []
        for _ in range(count):
            h = B // 2
            calls.append((g.insert, e[ai:ai + h]))
            calls.append((g.delete, present[pi:pi + h]))
            ai += h
            pi += h
        return calls

    out["mix_1e7"] = timed(mixed(B7, 3))
    out["mix_1e6"] = timed(mixed(B6, 10))
    out["ins_1e6"] = timed([(g.insert, e[ai + j * B6:ai + (j + 1) * B6]) for j in range(5)])
    ai += 5 * B6
    out["del_1e6"] = timed([(g.delete, present[pi + j * B6:pi + (j + 1) * B6]) for j in range(5)])
    pi += 5 * B6
    # Del at 1e7: everything still present
    rest = torch.cat([present[pi:], e[k:ai]])
    out["del_1e7"] = timed([(g.delete, rest[s:s + B7]) for s in range(0, rest.shape[0], B7)])
    out["empty_after_del"] = bool(int(g.levels().max()) == 0 and int(g.counters()[0].max()) == 0)
    g.close()
    del e, present, rest
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
            "config": {"workload": f"Chung-Lu n={n}, m={m}, exponent 2.1 (generated on the device, "
                                   f"{t_gen:.1f} s); grid {side}x{side} with 10% diagonals",
                       "value_is": "Ins protocol at batch 1e7 while loading 90% of the edges"},
            "chung_lu": out, "grid": grid}
    print(json.dumps(line), flush=True)


def run_batched(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    torch.cuda.set_device(0)
    ns, pre, rnds = make_batched(args.graphs, args.rounds)
    e0, o0 = P.PLDSSet.pack([(p_, np.zeros((0, 2), np.int32)) for p_ in pre])
    pre_dev = (torch.from_numpy(e0).cuda(), o0)
    packed = [P.PLDSSet.pack(r) for r in rnds]
    dev = [(torch.from_numpy(e).cuda(), o) for e, o in packed]
    upd = [int(o[-1]) for _, o in packed]
    w = min(args.warmup, args.rounds - 1)

    def timed_set(tuning):
        """Preload, warm-up rounds, then the timed rounds; returns (seconds, set)."""
        S = P.PLDSSet(ns)
        if tuning:
            S.tune(**tuning)
        S.update(*pre_dev)
        for r in range(w):
            S.update(*dev[r])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in range(w, args.rounds):
            S.update(*dev[r])
        torch.cuda.synchronize()
        return time.perf_counter() - t0, S

    # knobs picked by the autotuner on the preload and warm-up rounds only
    tuning = None
    t_tune = 0.0
    if not args.no_autotune and w > 0:
        probe = P.PLDSSet(ns)
        t0 = time.perf_counter()
        tuning = probe.autotune([pre_dev] + dev[:w], timed_from=1, max_trials=args.tune_trials)
        t_tune = time.perf_counter() - t0
        probe.close()
    dt_default, S0 = timed_set(None)
    S0.close()
    dt, S = timed_set(tuning)
    lat = dt / (args.rounds - w)
    batched = sum(upd[w:]) / dt
    # the plain form: one synchronous insert and delete call per graph, graphs one after another
    G = [P.PLDS(n) for n in ns]
    for g, p_ in zip(G, pre):
        g.insert(torch.from_numpy(p_).cuda())
    for r in range(w):
        for g, (ins, dele) in zip(G, rnds[r]):
            g.insert(torch.from_numpy(ins).cuda())
            g.delete(torch.from_numpy(dele).cuda())
    nplain = min(args.rounds - w, args.plain_rounds)
    devr = [[(torch.from_numpy(i_).cuda(), torch.from_numpy(d_).cuda()) for i_, d_ in rnds[r]]
            for r in range(w, w + nplain)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for rr in devr:
        for g, (ins, dele) in zip(G, rr):
            g.insert(ins)
            g.delete(dele)
    torch.cuda.synchronize()
    dtp = time.perf_counter() - t0
    plain = sum(upd[w:w + nplain]) / dtp
    same = all(np.array_equal(a.levels(), b.levels()) for a, b in zip(S.graphs, G)) if nplain == args.rounds - w else None
    line = {"metric": "edge updates/s, batched form (one launch per round of batches)", "value": batched,
            "unit": UNIT, "n_gpus": 1, "steps": args.rounds - w, "warmup": w, "ms_per_step": 1e3 * lat,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "form": "batched",
            "config": {"workload": f"{args.graphs} Chung-Lu graphs, n log-uniform [1e3,1e5], exponent U[2.1,2.8], "
                                   f"avg degree U[4,32], half preloaded, {args.rounds} mixed rounds of 1-10% of edges",
                       "total_vertices": int(sum(ns)), "updates_per_round": int(np.mean(upd))},
            "plain_loop": {"value": plain, "unit": UNIT, "rounds_timed": nplain,
                           "ms_per_round": 1e3 * dtp / nplain},
            "speedup_vs_plain": batched / plain, "levels_equal_plain": same,
            "autotune": {"knobs": tuning, "seconds": t_tune, "trials_max": args.tune_trials,
                         "sample": "preload + warm-up rounds (untimed)",
                         "default_knobs_updates_per_s": sum(upd[w:]) / dt_default}}
    print(json.dumps(line), flush=True)


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


def run_serving(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds as P
    torch.cuda.set_device(0)
    n, m = args.serve_n, args.serve_m
    e = W.chung_lu(n, m, 2.2, seed=1)
    pre, reqs = make_serving_stream(e, args.requests)
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
    for form, merge in (("served", -1), ("served_unmerged", 0)):
        g = preloaded()
        sv = P.Server(g, slots=args.slots, max_batch=2_000_000, merge_max_edges=merge)
        t0 = time.monotonic_ns()
        for op, b in pinned:
            if op == 2:
                sv.submit(2, out=qout.numpy())
            else:
                sv.submit(op, edges=b)
        sv.drain()
        done = sv.poll(4096)
        sv.close()
        g.close()
        span = (max(r["done_ns"] for r in done) - t0) * 1e-9
        results[f"{form}_capacity_updates_per_s"] = upd_total / span
        results[f"{form}_device_batches_back_to_back"] = sum(r["batch_first"] == r["ticket"] for r in done)

    def pct(x, q):
        return float(np.percentile(np.asarray(x) * 1e3, q))

    for load in (0.7, 0.9):
        rate = load * len(reqs) / cap_s
        rng = np.random.default_rng(99)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
        for form in ("plain", "served", "served_unmerged"):
            g = preloaded()
            lat = np.zeros(len(reqs))
            sizes = []
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
                sv = P.Server(g, slots=args.slots, max_batch=2_000_000,
                              merge_max_edges=-1 if form == "served" else 0)
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
            results[f"{form}@{int(load * 100)}%"] = {
                "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "mean_ms": float(lat.mean() * 1e3),
                "updates_per_s": upd_total / span, "makespan_s": span,
                **({"device_batches": len(sizes), "max_requests_per_batch": int(max(sizes))} if sizes else {})}
    best = results["served@90%"]
    line = {"metric": "edge updates/s and p50/p99 batch latency, serving form (device-resident request loop)",
            "value": results["served_capacity_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": len(reqs),
            "warmup": 0, "p50_ms_at_90pct": best["p50_ms"], "p99_ms_at_90pct": best["p99_ms"],
            "plain": {"capacity_updates_per_s": results["plain_capacity_updates_per_s"],
                      "p50_ms_at_90pct": results["plain@90%"]["p50_ms"],
                      "p99_ms_at_90pct": results["plain@90%"]["p99_ms"]},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "form": "serving",
            "config": {"workload": f"Chung-Lu n={n}, m={e.shape[0]}, exponent 2.2, 90% preloaded; "
                                   f"{len(reqs)} requests, sizes log-uniform [10,1e6], 50/50 Ins/Del, "
                                   "coreness query every 20 batches, Poisson arrivals at 70% and 90% of "
                                   "the plain form's capacity; inputs in pinned host memory; "
                                   "served = continuous batching (merged runs, logged schedule), "
                                   "served_unmerged = same loop with unchanged batch boundaries",
                       "slots": args.slots, "updates": upd_total},
            "results": results}
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

    def run_steps(g, k0, count, host=False, pinned=None, core_h=None):
        upd, recs = 0, []
        for k in range(k0, k0 + count):
            kind, a, b = steps[k % len(steps)]
            if host:
                src = pinned[kind][a:b]
            else:
                src = (ins_d if kind == "ins" else del_d)[a:b]
            (g.insert if kind == "ins" else g.delete)(src)
            recs.append(g.stats())
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
    with ClockSampler(local) as clk:
        ev0.record()
        upd, recs = run_steps(g, args.warmup, args.steps)
        ev1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = g.stats()["launches"] - launches0
    g.close()
    upd_all, t_max_s = whole_job(dist, upd, ms / 1e3, "cuda")
    t_max = t_max_s * 1e3
    value = upd_all / t_max_s

    # roofline of the batch kernel: algorithmic bytes / event-timed kernel duration
    kern_ns = sum(r["kernel_ns"] for r in recs)
    abytes = sum(algo_bytes(r) for r in recs)
    achieved = abytes / (kern_ns / 1e9) / 1e9 if kern_ns else None
    peak, peak_src = measured_peaks()
    traffic = None
    if NCU_TRAFFIC["kernel_sha"] == kernel_sha() and NCU_TRAFFIC["dram_per_algo_byte"]:
        traffic = NCU_TRAFFIC["dram_per_algo_byte"] * abytes / len(recs)
    if args.dump_recs:  # per timed step: the batch kernel's algorithmic bytes (matches ncu launch lists)
        with open(args.dump_recs, "w") as f:
            json.dump([{"algo_bytes": algo_bytes(r), "kernel_ns": r["kernel_ns"], "launches": r["launches"],
                        "valid": r["valid"]} for r in recs], f)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "kernel": "k_batch_grid", "peak_source": peak_src,
            "kernel_ms_per_launch": kern_ns / 1e6 / len(recs),
            "algo_bytes_per_launch": abytes / len(recs)}

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

    # per-batch latency of the timed steps (kernel time of each call)
    lat_ms = [r["kernel_ns"] / 1e6 for r in recs]
    protocols = None
    if world == 1 and not args.no_protocols:
        protocols = run_protocols(P, n, e, ins_d, del_d)
        # the paper's optimised variant: ceil(log_{1+delta} m / 50) levels per group
        lg_opt = P.opt_levels_per_group(int(e.shape[0]))
        protocols["plds_opt"] = {"levels_per_group": lg_opt,
                                 **run_protocols(P, n, e, ins_d, del_d, levels_per_group=lg_opt,
                                                 sizes=(1_000_000,))}

    phases = {}
    for kind in ("ins", "del"):
        sel = [(r, steps[(args.warmup + i) % len(steps)]) for i, r in enumerate(recs)
               if steps[(args.warmup + i) % len(steps)][0] == kind]
        if sel:
            ns = sum(r["kernel_ns"] for r, _ in sel)
            phases[kind] = {"steps": len(sel), "updates_per_s_kernel": sum(s[2] - s[1] for _, s in sel) / (ns / 1e9)}

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
        "phases": phases,
        "batch_latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                             "of": "batch kernel time of each timed step"},
        "protocols": protocols,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
