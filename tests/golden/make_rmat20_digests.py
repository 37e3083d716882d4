"""Write the per-batch oracle digests of the R-MAT scale-20 protocols at batch 10^6.

Calls only the sequential CPU oracle (oracle/) and the seeded workload generators:
no value here comes from the CUDA library.  For every batch of

  * Ins: all edges of R-MAT(20, 16, .57/.19/.19/.05, seed 1) from the empty graph,
    shuffle seed 11, batches of 10^6;
  * Del: then all of them, shuffle seed 12, batches of 10^6;
  * Mix: a fresh graph preloaded with 90 % of the edges (mix_stream seed 3, batches
    of 10^6), then 10 mixed batches (5*10^5 insertions from the absent edges, then
    5*10^5 deletions of present ones, Algorithm 1's order),

it records SHA-256 digests of the level array and of the counters deg, up and up*
(int32, little-endian) and the batch's work counts.  A fingerprint of the edge
streams lets a reader tell a different stream from different levels.

  python tests/golden/make_rmat20_digests.py   # ~15-20 min on one core
"""
from __future__ import annotations

import hashlib
import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import oracle as O  # noqa: E402
from paper_2106_03824_gb300 import workloads as W  # noqa: E402

B = 1_000_000
OUT = Path(__file__).resolve().parent / "rmat20_B1e6_digests.json"


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def record(o: O.OraclePLDS, kind: str, size: int) -> dict:
    st = o.stats()
    d, u, s = o.counters()
    return {"kind": kind, "size": size, "levels": digest(o.levels()), "counters": digest(d, u, s),
            **{k: st[k] for k in ("valid", "rounds", "moves", "visits", "dl_evals", "dl_visits")}}


def main():
    t0 = time.time()
    e = W.rmat(20, 16, seed=1)
    ins = W.shuffled(e, 11)
    dele = W.shuffled(e, 12)
    n = 1 << 20
    out = {"cite": "Algorithms 1-3 (batch insertion and deletion rounds), Invariants 1-2; "
                   "Experiments section: Ins/Del/Mix protocols; written by this script from oracle/ only",
           "graph": "R-MAT scale 20, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05), seed 1",
           "n": n, "m": int(e.shape[0]), "batch": B, "delta": 0.4, "lambda": 3,
           "stream_sha256": {"edges": digest(e), "ins": digest(ins), "del": digest(dele)},
           "digest": "sha256 over int32 little-endian arrays: levels; deg||up||up*"}
    o = O.OraclePLDS(n)
    recs = []
    for s0 in range(0, ins.shape[0], B):
        b = ins[s0:s0 + B]
        assert o.insert(b) == 0
        recs.append(record(o, "ins", int(b.shape[0])))
        print(f"ins {s0 // B} {time.time() - t0:.0f}s", flush=True)
    for s0 in range(0, dele.shape[0], B):
        b = dele[s0:s0 + B]
        assert o.delete(b) == 0
        recs.append(record(o, "del", int(b.shape[0])))
        print(f"del {s0 // B} {time.time() - t0:.0f}s", flush=True)
    out["ins_del"] = recs
    o.close()
    pre, mixes = W.mix_stream(e, B, 10, load=0.9, seed=3)
    out["stream_sha256"]["mix_pre"] = digest(pre)
    o = O.OraclePLDS(n)
    recs = []
    for s0 in range(0, pre.shape[0], B):
        b = pre[s0:s0 + B]
        assert o.insert(b) == 0
        recs.append(record(o, "pre", int(b.shape[0])))
    print(f"mix preload {time.time() - t0:.0f}s", flush=True)
    for a, b in mixes:
        assert o.insert(a) == 0
        recs.append(record(o, "ins", int(a.shape[0])))
        assert o.delete(b) == 0
        recs.append(record(o, "del", int(b.shape[0])))
    out["mix"] = recs
    out["oracle_seconds"] = round(time.time() - t0, 1)
    OUT.write_text(json.dumps(out, indent=1) + "\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f}s")


if __name__ == "__main__":
    main()
