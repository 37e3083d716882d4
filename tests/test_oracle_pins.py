"""Pins of the CPU oracle to things other than itself (CPU only).

Each test names the paper passage or mathematical fact it checks:
printed worked-example values, closed forms, brute force on tiny graphs, the
global-fixpoint restatement of the batch rules, invariants and the approximation
bound.  ``test_oracle_mutants.py`` re-runs this file against deliberately broken
copies of the oracle and expects it to fail for each.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03824_gb300 import workloads as W
import _ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------
# Threshold tables (Invariants 1 and 2; group size)
# ----------------------------------------------------------------------------

def test_printed_cutoffs_insertion_example():
    """Insertion example: cutoff 3 in group 0 and 4.2 in group 1 (delta=0.4, lambda=3)."""
    g = _load("insertion_example.json")["printed_cutoffs"]
    T = O.tables(1000, 0.4, 3.0)
    assert T["upmax"][0] == g["group0"] == 3
    assert T["upmax"][1] == g["group1_int"] == math.floor(g["group1_real"])


def test_printed_lower_bound_deletion_example():
    """Deletion example: the Invariant-2 bound for group 1 is (1+1)^1 = 2 at delta=1."""
    g = _load("deletion_example.json")
    T = O.tables(1000, 1.0, 3.0)
    assert T["dnmin"][1] == g["printed_lower_bound_group1"] == 2
    assert T["dnmin"][0] == 1


@pytest.mark.parametrize("n", [1, 2, 3, 16, 17, 1000, 1 << 20])
def test_closed_form_delta_one(n):
    """delta=1: (1+delta)^i = 2^i exactly, so upmax = 3*2^i, dnmin = 2^i, t = ceil(log2 n)."""
    T = O.tables(n, 1.0, 3.0)
    t = 0 if n == 1 else (n - 1).bit_length()
    assert T["t"] == t
    assert T["G"] == t + 1
    assert T["Lg"] == 4 * max(1, t)
    assert T["K"] == (t + 1) * 4 * max(1, t)
    for i in range(T["G"]):
        assert T["upmax"][i] == min(3 * 2 ** i, n)
        assert T["dnmin"][i] == min(2 ** i, n)


def test_closed_form_lambda_one_delta_half():
    """lambda=1, delta=1/2: (2+3)(3/2)^i; check the floor/ceil defining inequalities."""
    n = 10**6
    T = O.tables(n, 0.5, 1.0)
    for i in range(T["G"]):
        x5 = 5 * 3 ** i
        den = 2 ** i
        u = int(T["upmax"][i])
        if u < n:
            assert u * den <= x5 < (u + 1) * den
        else:
            assert x5 >= n * den
        d = int(T["dnmin"][i])
        if d < n:
            assert (d - 1) * den < 3 ** i <= d * den
        else:
            assert 3 ** i >= (n - 1) * den


def test_t_is_smallest_power_reaching_n():
    """t = ceil(log_{1.4} n) taken exactly: 7^t >= n 5^t and 7^(t-1) < n 5^(t-1)."""
    for n in [2, 3, 10, 12, 10**4, 2**20, 4_800_000, 24_000_000, 41_700_000]:
        t = O.tables(n)["t"]
        assert 7 ** t >= n * 5 ** t
        assert 7 ** (t - 1) < n * 5 ** (t - 1)


def test_tables_agree_with_fractions_module():
    """Random rational delta/lambda (denominator 10^6): same integers as Python Fractions."""
    rng = np.random.default_rng(5)
    for _ in range(25):
        delta = float(rng.choice([0.2, 0.4, 0.8, 1.6, 3.2, 6.4, round(rng.uniform(0.15, 3), 6)]))
        lam = float(rng.choice([3, 6, 12, 24, 48, 96, round(rng.uniform(0.5, 50), 6)]))
        n = int(rng.integers(1, 5_000_000))
        T = O.tables(n, delta, lam)
        R = _ref.fraction_tables(n, delta, lam)
        assert T["t"] == R["t"] and T["K"] == R["K"]
        assert list(T["upmax"]) == R["upmax"]
        assert list(T["dnmin"]) == R["dnmin"]


def test_bad_parameters_rejected():
    for args in [(0, 0.4, 3.0), (10, 0.0, 3.0), (10, -1.0, 3.0), (10, 0.4, 0.0), (10, 0.4, -2.0)]:
        with pytest.raises(ValueError):
            O.tables(*args)


# ----------------------------------------------------------------------------
# Exact coreness (Matula-Beck) against the definition
# ----------------------------------------------------------------------------

def _cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


@pytest.mark.parametrize("name,n,edges,expect", [
    ("K6", 6, [(i, j) for i in range(6) for j in range(i + 1, 6)], [5] * 6),
    ("C7", 7, _cycle(7), [2] * 7),
    ("path5", 5, [(i, i + 1) for i in range(4)], [1] * 5),
    ("star", 8, [(0, i) for i in range(1, 8)], [1] * 8),
    ("K34", 7, [(i, j) for i in range(3) for j in range(3, 7)], [3] * 7),
    ("empty", 4, [], [0] * 4),
    ("petersen", 10, [(i, (i + 1) % 5) for i in range(5)] + [(i, i + 5) for i in range(5)]
     + [(5 + i, 5 + (i + 2) % 5) for i in range(5)], [3] * 10),
    ("K4+tail", 6, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3), (3, 4), (4, 5)],
     [3, 3, 3, 3, 1, 1]),
])
def test_exact_coreness_closed_forms(name, n, edges, expect):
    assert list(O.exact_coreness(n, edges)) == expect


def test_exact_coreness_matches_brute_force():
    rng = np.random.default_rng(7)
    for trial in range(60):
        n = int(rng.integers(2, 13))
        m = int(rng.integers(0, n * (n - 1) // 2 + 1))
        e = W.erdos_renyi(n, m, seed=trial)
        assert list(O.exact_coreness(n, e)) == _ref.brute_coreness(n, e)


# ----------------------------------------------------------------------------
# Coreness estimate (Definition "Coreness Estimate")
# ----------------------------------------------------------------------------

def test_coreness_estimate_paper_example():
    """Vertex on level 4 with 3-level groups: largest completed group is 0, estimate 1."""
    ex = _load("deletion_example.json")["coreness_example"]
    h = O.OraclePLDS(6, 1.0, 3.0, levels_per_group=3)
    h.add_edges_raw([(0, 1)])
    h.set_level(0, ex["level"])
    assert h.coreness_exponent()[0] == 0
    assert h.coreness()[0] == ex["estimate"]


def test_coreness_estimate_group_boundaries():
    """Top level of group i, (i+1)L-1, gives (1+delta)^i; one level lower gives i-1."""
    h = O.OraclePLDS(40, 0.4, 3.0, levels_per_group=5)
    h.add_edges_raw([(0, 1), (2, 3)])
    for i in range(1, 6):
        h.set_level(0, (i + 1) * 5 - 1)
        h.set_level(2, (i + 1) * 5 - 2)
        g = h.coreness_exponent()
        assert g[0] == i and g[2] == i - 1
        assert h.coreness()[0] == pytest.approx(1.4 ** i, rel=1e-14)
    g = h.coreness_exponent()
    assert g[5] == -1 and h.coreness()[5] == 0.0  # isolated vertex: estimate 0


# ----------------------------------------------------------------------------
# Worked examples (Algorithms 2 and 3)
# ----------------------------------------------------------------------------

def _stage(ex):
    names = ex["names"]
    idx = {k: i for i, k in enumerate(names)}
    h = O.OraclePLDS(len(names), ex["delta"], ex["lambda"], ex["levels_per_group"])
    assert h.add_edges_raw([(idx[a], idx[b]) for a, b in ex["edges"]]) == 0
    for k, l in ex["levels"].items():
        assert h.set_level(idx[k], l) == 0
    assert h.check() == 0, "staged example must satisfy both invariants"
    batch = [(idx[a], idx[b]) for a, b in ex["batch"]]
    expect = np.array([ex["expected_levels"][k] for k in names])
    return h, batch, expect


def test_insertion_worked_example():
    ex = _load("insertion_example.json")
    h, batch, expect = _stage(ex)
    assert h.insert(batch) == 0
    assert list(h.levels()) == list(expect)
    s = h.stats()
    assert s["rounds"] == ex["expected_rounds"] and s["moves"] == ex["expected_moves"]
    assert h.check() == 0


def test_deletion_worked_example():
    ex = _load("deletion_example.json")
    h, batch, expect = _stage(ex)
    assert h.delete(batch) == 0
    assert list(h.levels()) == list(expect)
    s = h.stats()
    assert s["rounds"] == ex["expected_rounds"] and s["moves"] == ex["expected_moves"]
    assert s["dl_evals"] == ex["expected_dl_evals"]
    assert s["max_vertex_moves"] == 1
    assert h.check() == 0


# ----------------------------------------------------------------------------
# Batch rules against the global-fixpoint restatement (tiny graphs)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("delta,lam,lpg", [(0.4, 3.0, 0), (0.4, 3.0, 3), (1.0, 3.0, 3),
                                           (0.2, 1.0, 2), (1.6, 12.0, 0)])
def test_rules_match_global_fixpoint(delta, lam, lpg):
    """Both insertion procedures -- one level a round (Algorithm 2) and the jump mode
    (violators straight to their targets) -- land on the global fixpoint's levels;
    the jump mode never makes more moves (each of its moves climbs at least one level
    of the same total climb)."""
    rng = np.random.default_rng(int(delta * 100 + lam + lpg))
    for trial in range(12):
        n = int(rng.integers(4, 26))
        allp = _ref.all_pairs(n)
        h = O.OraclePLDS(n, delta, lam, lpg)
        hj = O.OraclePLDS(n, delta, lam, lpg, flags=O.JUMP)
        g = _ref.GlobalPLDS(n, delta, lam, lpg)
        present = set()
        for step in range(10):
            if rng.random() < 0.6 or not present:
                k = int(rng.integers(1, max(2, len(allp) // 3)))
                pick = [allp[i] for i in rng.choice(len(allp), size=k, replace=False)]
                assert h.insert(pick) == 0 and hj.insert(pick) == 0
                assert hj.stats()["moves"] <= h.stats()["moves"]
                g.insert(pick)
                present |= set(pick)
            else:
                pl = sorted(present)
                k = int(rng.integers(1, len(pl) + 1))
                pick = [pl[i] for i in rng.choice(len(pl), size=k, replace=False)]
                assert h.delete(pick) == 0 and hj.delete(pick) == 0
                g.delete(pick)
                present -= set(pick)
            assert list(h.levels()) == g.level, (trial, step)
            assert list(hj.levels()) == g.level, (trial, step)
            assert h.check() == 0 and hj.check() == 0


def test_jump_mode_hand_example():
    """n = 12, delta = 0.4, lambda = 3: t = 8 (1.4^7 < 12 <= 1.4^8), 32 levels a group,
    UPMAX = floor(3 * 1.4^i) = 3, 4, 5, 8, 11, 12, ... and DNMIN = ceil(1.4^i) = 1, 2, 2,
    3, 4, 6, ...  A clique on vertices 1..11 sits on level 160 (group 5: up 10 <= 12,
    up* 10 >= DNMIN[4] = 4).  Inserting (0, 1..9) leaves vertex 0 on level 0 with up 9
    > 3.  Its target is the first level whose group allows 9 up-neighbours, group 4
    (UPMAX 11) from level 128 on, below the clique: Algorithm 2 climbs there in 128
    rounds of one move, the jump mode in one."""
    T = O.tables(12)
    assert T["t"] == 8 and T["Lg"] == 32
    assert list(T["upmax"][:6]) == [3, 4, 5, 8, 11, 12] and list(T["dnmin"][:6]) == [1, 2, 2, 3, 4, 6]
    clique = [(u, v) for u in range(1, 12) for v in range(u + 1, 12)]
    for flags, rounds in ((0, 128), (O.JUMP, 1)):
        h = O.OraclePLDS(12, flags=flags)
        h.add_edges_raw(clique)
        for v in range(1, 12):
            h.set_level(v, 160)
        assert h.check() == 0
        assert h.insert([(0, v) for v in range(1, 10)]) == 0
        lv = h.levels()
        assert lv[0] == 128 and all(lv[1:] == 160)
        s = h.stats()
        assert s["rounds"] == rounds and s["moves"] == rounds and s["max_vertex_moves"] == 128
        assert h.check() == 0


# ----------------------------------------------------------------------------
# Invariants, move directions and the approximation bound
# ----------------------------------------------------------------------------

def _bound_ok(h, n, delta, lam):
    core = O.exact_coreness(n, h.edges())
    g = h.coreness_exponent()
    d = _ref.rational(delta)
    lm = _ref.rational(lam)
    base = 1 + d
    cprime = (2 + Fraction(3) / lm) * base
    for gi, k in zip(g, core):
        gi, k = int(gi), int(k)
        if gi < 0 or k == 0:
            if not (gi < 0 and k == 0):
                return False
            continue
        khat = base ** gi
        if not (k <= cprime * khat and khat <= cprime * k):
            return False
    return True


def test_tiny_graphs_invariants_bound_and_brute_force():
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(2, 13))
        allp = _ref.all_pairs(n)
        h = O.OraclePLDS(n)
        present = set()
        for step in range(8):
            if rng.random() < 0.65 or not present:
                k = int(rng.integers(1, len(allp) + 1))
                pick = [allp[i] for i in rng.choice(len(allp), size=k, replace=False)]
                assert h.insert(pick) == 0
                assert h.stats()["dir_error"] == 0
                present |= set(pick)
            else:
                pl = sorted(present)
                k = int(rng.integers(1, len(pl) + 1))
                pick = [pl[i] for i in rng.choice(len(pl), size=k, replace=False)]
                assert h.delete(pick) == 0
                s = h.stats()
                assert s["dir_error"] == 0 and s["max_vertex_moves"] <= 1
                present -= set(pick)
            assert h.check() == 0
            e = h.edges()
            assert sorted(map(tuple, e.tolist())) == sorted(present)
            assert list(O.exact_coreness(n, e)) == _ref.brute_coreness(n, e)
            assert _bound_ok(h, n, 0.4, 3.0)


def test_small_config_invariants_and_bound_every_batch():
    """Chung-Lu n=10^4, m=5*10^4, gamma=2.5: 50 Ins batches then 50 Del batches of 1000."""
    n = 10_000
    e = W.chung_lu(n, 50_000, 2.5, seed=1)
    h = O.OraclePLDS(n)
    for b in W.batches(W.shuffled(e, 11), 1000):
        assert h.insert(b) == 0
        assert h.check() == 0
        assert h.stats()["dir_error"] == 0
        assert _bound_ok(h, n, 0.4, 3.0)
    for b in list(W.batches(W.shuffled(h.edges(), 12), 1000))[:50]:
        assert h.delete(b) == 0
        s = h.stats()
        assert s["max_vertex_moves"] <= 1 and s["dir_error"] == 0
        assert h.check() == 0
        assert _bound_ok(h, n, 0.4, 3.0)


def test_counters_by_definition_consistent():
    """deg = sum of up contributions: up(v) <= up*(v) <= deg(v) for every v."""
    e = W.chung_lu(2000, 9000, 2.3, seed=4)
    h = O.OraclePLDS(2000)
    for b in W.batches(e, 1500):
        h.insert(b)
    d, u, s = h.counters()
    assert (u <= s).all() and (s <= d).all()
    assert d.sum() == 2 * h.edges().shape[0]


# ----------------------------------------------------------------------------
# Batch preprocessing (framework section: unique, valid updates)
# ----------------------------------------------------------------------------

def test_preprocessing_filters_and_counts():
    n = 50
    h = O.OraclePLDS(n)
    base = W.erdos_renyi(n, 120, seed=2)
    noisy = W.noisy_batch(base, n, seed=3, self_loops=7, dups=25, reversed_frac=0.3)
    assert h.insert(noisy) == 0
    s = h.stats()
    assert s["self_loops"] == 7 and s["duplicates"] == 25 and s["valid"] == base.shape[0]
    assert h.edges().shape[0] == base.shape[0]
    lv = h.levels().copy()
    assert h.insert(base[:10]) == 0          # already present: filtered, nothing moves
    assert h.stats()["filtered"] == 10 and h.stats()["valid"] == 0
    assert list(h.levels()) == list(lv)
    absent = [(a, b) for a in range(n) for b in range(a + 1, n)
              if (a, b) not in set(map(tuple, base.tolist()))][:5]
    assert h.delete(absent) == 0             # absent: filtered
    assert h.stats()["filtered"] == 5 and h.stats()["valid"] == 0
    assert h.insert(np.zeros((0, 2), np.int32)) == 0   # empty batch is a no-op
    assert list(h.levels()) == list(lv)


def test_out_of_range_rejected_before_any_change():
    n = 20
    h = O.OraclePLDS(n)
    h.insert(W.erdos_renyi(n, 40, seed=9))
    lv = h.levels().copy()
    m = h.edges().shape[0]
    assert h.insert([(0, 1), (2, n)]) == O.ORC_EINVAL
    assert h.insert([(-1, 3)]) == O.ORC_EINVAL
    assert h.delete([(0, 1), (n + 5, 1)]) == O.ORC_EINVAL
    assert list(h.levels()) == list(lv) and h.edges().shape[0] == m


# ----------------------------------------------------------------------------
# PLDSOpt levels per group (experiments section, "Evaluated Algorithms")
# ----------------------------------------------------------------------------

def test_opt_levels_per_group_livejournal_example():
    """The paper's livejournal example (m = 42,851,237): log_1.4(m) = 52.2, so the
    formula gives ceil(1.04) = 2 at delta = 0.4; it gives 1 only from delta ~ 0.4212
    up (the text's "1 for all delta < 0.42" has the inequality reversed), and 1 across
    the [0.8, 6.4] range where the paper reports flat PLDSOpt curves."""
    m = 42_851_237
    assert O.opt_levels_per_group(m, 0.4) == 2
    assert O.opt_levels_per_group(m, 0.4211) == 2
    assert O.opt_levels_per_group(m, 0.4212) == 1
    for d in (0.43, 0.8, 1.6, 3.2, 6.4):
        assert O.opt_levels_per_group(m, d) == 1


def test_opt_levels_per_group_closed_forms():
    # 1.1^50 = 117.39..., 1.1^100 = 13780.61...
    assert O.opt_levels_per_group(117, 0.1) == 1
    assert O.opt_levels_per_group(118, 0.1) == 2
    assert O.opt_levels_per_group(13_780, 0.1) == 2
    assert O.opt_levels_per_group(13_781, 0.1) == 3
    # 2^50 > 2^32: one level per group for every m at delta = 1
    assert O.opt_levels_per_group(2**32 - 1, 1.0) == 1
    # log <= 0: at least one level
    assert O.opt_levels_per_group(0, 0.4) == 1
    assert O.opt_levels_per_group(1, 0.4) == 1
    with pytest.raises(ValueError):
        O.opt_levels_per_group(2**32, 0.4)
    with pytest.raises(ValueError):
        O.opt_levels_per_group(-1, 0.4)


def test_opt_levels_per_group_against_logarithms():
    """Away from the boundaries, ceil(ln m / ln(1+delta) / 50) in floating point."""
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(400):
        d = float(rng.choice([0.05, 0.1, 0.2, 0.4, 0.8, 1.6]))
        m = int(np.exp(rng.uniform(0, np.log(2**32 - 1))))
        x = math.log(max(m, 1)) / math.log(1 + d) / 50
        if abs(x - round(x)) < 1e-6:
            continue
        assert O.opt_levels_per_group(m, d) == max(1, math.ceil(x)), (m, d)
        checked += 1
    assert checked > 350


# ----------------------------------------------------------------------------
# Low out-degree orientation (Section "O(alpha) Out-Degree Orientation", Algorithm 5)
# ----------------------------------------------------------------------------

def test_orientation_hand_example():
    """Triangle 0-1-2 plus edge 2-3, levels 3, 1, 1, 1: edges go from the lower level
    to the higher one, and on equal levels from the lower id to the higher id
    (Algorithm 5's flip conditions keep H[(u,v)] = 0, u < v, when levels are equal)."""
    h = O.OraclePLDS(4, 1.0, 3.0, levels_per_group=3)
    h.add_edges_raw([(0, 1), (1, 2), (0, 2), (2, 3)])
    for v, l in ((0, 3), (1, 1), (2, 1), (3, 1)):
        h.set_level(v, l)
    tails = h.orient([(0, 1), (1, 2), (0, 2), (2, 3), (3, 2), (0, 3), (1, 1), (0, 9)])
    assert list(tails) == [1, 1, 2, 2, 2, -1, -1, -1]
    assert list(h.out_degrees()) == [0, 2, 2, 0]


def _key_order(levels, u, v):
    return (levels[u], u) < (levels[v], v)


def test_orientation_acyclic_bounded_and_flips_by_brute_force():
    """On random batch sequences: every edge goes up the (level, id) order (so the
    orientation is acyclic), out-degree <= up-degree <= the level's Invariant-1
    cutoff, and F / J equal a brute-force comparison of the level arrays and edge
    sets before and after each batch."""
    rng = np.random.default_rng(21)
    n = 60
    allp = _ref.all_pairs(n)
    for trial in range(6):
        h = O.OraclePLDS(n)
        h.track(True)
        T = O.tables(n)
        present = set()
        for step in range(10):
            before_lv = h.levels().copy()
            before_e = set(map(tuple, h.edges().tolist()))
            if rng.random() < 0.6 or not present:
                pick = [allp[i] for i in rng.choice(len(allp), size=int(rng.integers(1, 120)), replace=False)]
                h.insert(pick)
                op = 0
            else:
                cur = sorted(present)
                pick = [cur[i] for i in rng.choice(len(cur), size=int(rng.integers(1, len(cur) + 1)), replace=False)]
                h.delete(pick)
                op = 1
            lv = h.levels()
            after_e = set(map(tuple, h.edges().tolist()))
            present = after_e
            deg, up, _ = h.counters()
            out = h.out_degrees()
            for (u, v) in after_e:
                t = h.orient([(u, v)])[0]
                assert t == (u if _key_order(lv, u, v) else v)
            assert np.all(out <= up)
            assert np.all(out <= np.asarray(T["upmax"])[lv // T["Lg"]])
            assert out.sum() == len(after_e)
            expect_f = sorted((u, v) if _key_order(before_lv, u, v) else (v, u)
                              for (u, v) in (before_e & after_e)
                              if _key_order(before_lv, u, v) != _key_order(lv, u, v))
            assert [tuple(x) for x in h.flips().tolist()] == expect_f
            changed = (after_e - before_e) if op == 0 else (before_e - after_e)
            ref_lv = lv if op == 0 else before_lv
            expect_j = sorted((u, v) if _key_order(ref_lv, u, v) else (v, u) for (u, v) in changed)
            assert [tuple(x) for x in h.oriented_updates().tolist()] == expect_j
        h.close()


def test_heuristic_coefficient_tables():
    """Heuristic parameters (experiments section): 2 + 3/lambda replaced by 1.1, so
    upmax[i] = floor(1.1 * 1.4^i): 1, 1, 2, 3, 4, 5 (1.1 * 1.4^5 = 5.916...), and the
    Invariant-2 side is unchanged."""
    T = O.tables(1000, 0.4, 3.0, flags=O.HEURISTIC)
    assert list(T["upmax"][:6]) == [1, 1, 2, 3, 4, 5]
    assert list(T["dnmin"]) == list(O.tables(1000, 0.4, 3.0)["dnmin"])
    # lambda plays no part any more
    assert list(T["upmax"]) == list(O.tables(1000, 0.4, 96.0, flags=O.HEURISTIC)["upmax"])
    # the invariants still hold after every batch
    e = W.chung_lu(2000, 12_000, 2.3, seed=4)
    h = O.OraclePLDS(2000, flags=O.HEURISTIC)
    for b in W.batches(W.shuffled(e, 1), 3000):
        assert h.insert(b) == 0
        assert h.check() == 0
    for b in W.batches(W.shuffled(e, 2), 3000):
        assert h.delete(b) == 0
        assert h.check() == 0


# ----------------------------------------------------------------------------
# Static (2+eps')-approximate k-core (Section "Static (2+eps)-Approximate k-Core",
# Algorithm 6)
# ----------------------------------------------------------------------------

def _static_graph(n, edges):
    h = O.OraclePLDS(n, 1.0, 3.0, levels_per_group=3)
    h.add_edges_raw(edges)
    return h


def test_static_worked_example():
    """The paper's example with eps = 1 (eps' = 4): v, w, a, b of degree 2 go to
    bucket ceil(log2 2) = 1 and get 2; u, x, y, z (a K4, one extra neighbour each)
    keep degree >= 3 after the first peel, stay in bucket 2 and get 4."""
    u, x, y, z, v, w, a, b = range(8)
    E = [(u, x), (u, y), (u, z), (x, y), (x, z), (y, z), (v, u), (v, w), (w, x), (a, y), (a, b), (b, z)]
    est, st = _static_graph(8, E).static_coreness(4.0)
    assert list(est) == [4, 4, 4, 4, 2, 2, 2, 2]
    thr, J = O.static_thresholds(8, 4.0)
    assert list(thr) == [1, 2, 4, 8]          # eps = (sqrt(25) - 3) / 2 = 1 exactly
    assert J == 2                             # delta = 2: ceil(log_3 8) = 2


def test_static_closed_forms():
    # a clique on k+1 vertices: all peeled together, estimate = (1+eps)^ceil(log_{1+eps} k)
    k = 9
    E = [(i, j) for i in range(k + 1) for j in range(i + 1, k + 1)]
    est, _ = _static_graph(k + 1, E).static_coreness(4.0)
    assert np.all(est == 16.0)               # ceil(log2 9) = 4
    # a star: leaves first (bucket 0), the centre drops to the clamp 1 and follows: all 1
    E = [(0, i) for i in range(1, 40)]
    est, st = _static_graph(40, E).static_coreness(1.0)
    assert np.all(est == 1.0) and st["outer"] == 1
    # isolated vertices: 0; a path: all 1
    est, _ = _static_graph(6, [(0, 1), (1, 2), (2, 3)]).static_coreness(1.0)
    assert list(est) == [1, 1, 1, 1, 0, 0]


def test_static_within_bound_of_exact():
    """Estimates are within 2 + eps' of the exact coreness both ways (and 0 exactly
    on isolated vertices), on power-law graphs and on all graphs of brute-force size."""
    for ep in (0.5, 1.0, 2.0, 4.0):
        for seed in range(4):
            for n, m, gam in ((1500, 12000, 2.2), (300, 6000, 2.1)):
                e = W.chung_lu(n, m, gam, seed=seed)
                est, _ = _static_graph(n, e).static_coreness(ep)
                core = O.exact_coreness(n, e).astype(np.float64)
                nz = core > 0
                assert np.array_equal(est == 0, ~nz)
                assert np.all(est[nz] <= (2 + ep) * core[nz]) and np.all(core[nz] <= (2 + ep) * est[nz])
    rng = np.random.default_rng(9)
    for trial in range(40):
        n = int(rng.integers(2, 11))
        allp = _ref.all_pairs(n)
        pick = [allp[i] for i in rng.choice(len(allp), size=int(rng.integers(1, len(allp) + 1)), replace=False)]
        core = np.asarray(_ref.brute_coreness(n, pick), np.float64)
        est, _ = _static_graph(n, pick).static_coreness(1.0)
        nz = core > 0
        assert np.array_equal(est == 0, ~nz)
        assert np.all(est[nz] <= 3 * core[nz]) and np.all(core[nz] <= 3 * est[nz])


def test_static_threshold_test_traced_example():
    """A traced run (eps' = 4: eps = 1, delta = 2, J = ceil(log_3 8) = 2, thresholds
    1, 2, 4, 8).  Degrees 1, 1, 4, 5, 5, 5, 4, 3 give buckets 0, 0, 2, 3, 3, 3, 2, 2.
    t = 0 peels {0, 1} (estimate 1); 4 and 5 drop to degree 4, bucket 2.  The next
    bucket fails the test 4 <= (2+1)*1, so t becomes 2: {2, 4, 5, 6, 7} are peeled at
    4, and 3 (degree 0 left, floored at the bucket t = 2) follows at 4.  Peeling
    bucket 2 still at t = 0 would have let 3 fall to bucket 0 (estimate 1)."""
    E = [(0, 5), (1, 4), (2, 3), (2, 4), (2, 6), (2, 7), (3, 4), (3, 5), (3, 6), (3, 7), (4, 5), (4, 6),
         (5, 6), (5, 7)]
    est, st = _static_graph(8, E).static_coreness(4.0)
    assert list(est) == [1, 1, 4, 4, 4, 4, 4, 4]
    assert st["outer"] == 2 and st["inner"] == 3
