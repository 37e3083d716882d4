"""Write the per-batch oracle digests of the first 10^8 updates of the large
configuration's insertion stream.

Calls only the sequential CPU oracle (oracle/) and the seeded workload generator:
no value here comes from the CUDA library.  The stream is the counter-based
Chung-Lu draw stream (workloads.ChungLuDraws: n = 41.7 M, m = 1.2 B, exponent
2.1, seed 1) that the large configuration loads its graph from, in its own batches
of 10^7 draws (raw pairs: repeats and self-loops are part of the stream and are
dropped by the batch rules).  After each of the first ten batches (10^8 updates)
it records SHA-256 digests of the level array and of deg||up||up* (int32,
little-endian) and the batch's work counts; a digest of the draws lets a reader
tell a different stream from different levels.

  python tests/golden/make_large_digests.py   # about an hour on one core, ~6 GB
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

N, M, GAMMA, SEED = 41_700_000, 1_200_000_000, 2.1, 1
B, NB = 10_000_000, 10
OUT = Path(__file__).resolve().parent / "chunglu41m_first1e8_digests.json"


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


def main():
    t0 = time.time()
    gen = W.ChungLuDraws(N, M, GAMMA, seed=SEED)
    out = {"cite": "Algorithm 2 (batch insertion rounds), Invariants 1-2; Experiments section: "
                   "insertion batches; written by this script from oracle/ only",
           "graph": f"counter-based Chung-Lu draws n={N}, m={M}, exponent {GAMMA}, seed {SEED}",
           "n": N, "m": M, "batch": B, "delta": 0.4, "lambda": 3,
           "digest": "sha256 over int32 little-endian arrays: levels; deg||up||up*; draws of each batch",
           "perm_sha256": digest(gen.perm), "cw_sha256": hashlib.sha256(gen.cw.astype("<i8").tobytes()).hexdigest()}
    o = O.OraclePLDS(N)
    recs = []
    for j in range(NB):
        b = gen.draws(j * B, B)
        t1 = time.time()
        assert o.insert(b) == 0
        st = o.stats()
        d, u, s = o.counters()
        recs.append({"kind": "ins", "start": j * B, "size": B, "draws": digest(b), "levels": digest(o.levels()),
                     "counters": digest(d, u, s), "oracle_seconds": round(time.time() - t1, 1),
                     **{k: st[k] for k in ("valid", "rounds", "moves", "visits", "dl_evals", "dl_visits")}})
        print(f"batch {j} valid {st['valid']} rounds {st['rounds']} {time.time() - t0:.0f}s", flush=True)
        out["ins"] = recs
        OUT.write_text(json.dumps(out, indent=1) + "\n")  # partial results survive an interruption
    o.close()
    out["seconds"] = round(time.time() - t0)
    OUT.write_text(json.dumps(out, indent=1) + "\n")
    print(f"wrote {OUT} in {out['seconds']}s")


if __name__ == "__main__":
    main()
