"""Bit-exact parity at the benchmark's own configuration (GPU).

R-MAT scale 20 (15.7 M edges, 2^20 vertices) at batches of 10^6, in the launch
configuration bench.py times (default tuning, device-resident batches): the Ins
protocol from the empty graph, the Del protocol after it, and the Mix protocol on
a 90 %-loaded graph.  After every batch the SHA-256 digests of the level array and
of deg||up||up* must equal the ones the sequential oracle wrote
(tests/golden/rmat20_B1e6_digests.json, made by make_rmat20_digests.py from
oracle/ only), and so must the batch's work counts.
"""
import hashlib
import json
from pathlib import Path

import numpy as np
import pytest

from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD = Path(__file__).resolve().parent / "golden" / "rmat20_B1e6_digests.json"
B = 1_000_000
COUNTS = ("valid", "rounds", "moves", "visits", "dl_evals", "dl_visits")


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a, dtype="<i4").tobytes())
    return h.hexdigest()


@pytest.fixture(scope="module")
def gold():
    return json.loads(GOLD.read_text())


@pytest.fixture(scope="module")
def stream(gold):
    e = W.rmat(20, 16, seed=1)
    ins, dele = W.shuffled(e, 11), W.shuffled(e, 12)
    # the oracle's stream and this one must be the same before levels can be compared
    assert digest(e) == gold["stream_sha256"]["edges"], "R-MAT generator gives another graph here"
    assert digest(ins) == gold["stream_sha256"]["ins"] and digest(dele) == gold["stream_sha256"]["del"]
    return e, ins, dele


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    return plds


def check(g, rec, what):
    d, u, s = g.counters()
    assert digest(g.levels()) == rec["levels"], f"{what}: levels differ from the oracle's"
    assert digest(d, u, s) == rec["counters"], f"{what}: counters differ from the oracle's"
    st = g.stats()
    for k in COUNTS:
        assert st[k] == rec[k], f"{what}: {k} gpu={st[k]} oracle={rec[k]}"


def test_rmat20_ins_del_every_batch(P, gold, stream):
    e, ins, dele = stream
    n = gold["n"]
    g = P.PLDS(n)
    ins_d, del_d = torch.from_numpy(ins).cuda(), torch.from_numpy(dele).cuda()
    recs = iter(gold["ins_del"])
    for s0 in range(0, ins.shape[0], B):
        g.insert(ins_d[s0:s0 + B])
        check(g, next(recs), f"ins batch {s0 // B}")
    for s0 in range(0, dele.shape[0], B):
        g.delete(del_d[s0:s0 + B])
        check(g, next(recs), f"del batch {s0 // B}")
    g.close()


def test_rmat20_mix_every_batch(P, gold, stream):
    e, _, _ = stream
    pre, mixes = W.mix_stream(e, B, 10, load=0.9, seed=3)
    assert digest(pre) == gold["stream_sha256"]["mix_pre"]
    g = P.PLDS(gold["n"])
    recs = iter(gold["mix"])
    pre_d = torch.from_numpy(pre).cuda()
    for s0 in range(0, pre.shape[0], B):
        g.insert(pre_d[s0:s0 + B])
        check(g, next(recs), f"preload batch {s0 // B}")
    for i, (a, b) in enumerate(mixes):
        g.insert(torch.from_numpy(a).cuda())
        check(g, next(recs), f"mix {i} insertions")
        g.delete(torch.from_numpy(b).cuda())
        check(g, next(recs), f"mix {i} deletions")
    g.close()
