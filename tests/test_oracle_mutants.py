"""The oracle's pins must catch plausible mistakes (CPU only).

Each case copies the oracle's C source, plants one mistake (a dropped term, a wrong
index or group, a skipped step), compiles the copy to a temporary library and runs
``test_oracle_pins.py`` against it in a subprocess; the pins must fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "plds_oracle.c")

MUTANTS = {
    # Invariant 1 tested against the next level's group instead of level l's
    "inv1_wrong_group": ("if (up_of(h, v) > h->T.upmax[gn(h, l)]) iv_push(&movers, v);",
                         "if (up_of(h, v) > h->T.upmax[gn(h, l + 1)]) iv_push(&movers, v);"),
    # up*(v) counted from level(v) instead of level(v)-1
    "upstar_off_by_one": ("int32_t c = 0, lv = h->level[v] - 1;",
                          "int32_t c = 0, lv = h->level[v];"),
    # desire-level: Invariant 2 checked one level too high
    "dl_index": ("int inv2 = (lp == 0) || hist[lp - 1] >= h->T.dnmin[gn(h, lp - 1)];",
                 "int inv2 = (lp == 0) || hist[lp] >= h->T.dnmin[gn(h, lp - 1)];"),
    # coreness estimate without the +1
    "coreness_formula": ("int32_t g = (h->level[v] + 1) / h->T.Lg - 1;\n        out[v] = g > 0 ? g : 0;",
                         "int32_t g = (h->level[v]) / h->T.Lg - 1;\n        out[v] = g > 0 ? g : 0;"),
    # Invariant-1 coefficient 2+2/lambda instead of 2+3/lambda
    "coefficient": ("(uint64_t)(2 * T->lnum + 3 * T->lden)", "(uint64_t)(2 * T->lnum + 2 * T->lden)"),
    # ceil of (1+delta)^i replaced by floor
    "dnmin_floor": ("T->dnmin[i] = (int32_t)bn_ceil_div_clamped(&pw, &qw, n, &err);",
                    "T->dnmin[i] = (int32_t)bn_floor_div_clamped(&pw, &qw, n, &err);"),
    # neighbours that now violate Invariant 2 never get their desire-level recomputed
    "no_dl_recompute": ("if (inv2_ok(h, w)) continue;\n                int32_t d = desire_level(h, w, hist);",
                        "if (1) continue;\n                int32_t d = desire_level(h, w, hist);"),
    # neighbours on level l+1 are never marked
    "no_marking": ("h->marked[w] = 1;\n                    iv_push(&bucket[l + 1], w);",
                   "iv_push(&bucket[l + 1], -1 < 0 ? v : w);"),
    # preprocessing keeps already-present edges
    "no_presence_filter": ("if (has_edge(h, u, v) != want_present) { h->st_filtered++; continue; }",
                           "if (0) { h->st_filtered++; continue; }"),
    # orientation ties broken from the higher id to the lower id
    "orient_tie": ("return lv[u] < lv[v] || (lv[u] == lv[v] && u < v);",
                   "return lv[u] < lv[v] || (lv[u] == lv[v] && u > v);"),
    # flips of the last batch compared against the levels after it on both sides
    "flips_no_snapshot": ("int before = goes_from(h->old_level, u, v), after = goes_from(h->level, u, v);",
                          "int before = goes_from(h->level, u, v), after = goes_from(h->level, u, v);"),
    # static k-core: estimate from the previous threshold (the prose's (1+eps)^(k-1))
    "static_estimate": ("est[v] = thr[bkt];", "est[v] = bkt > 0 ? thr[bkt - 1] : 0.5;"),
    # static k-core: the next bucket taken at the same threshold without the (2+eps) test
    "static_no_threshold_test": ("if (thr[next] <= (2.0 + eps) * thr[t]) bkt = next;", "if (1) bkt = next;"),
    # jump mode: the target taken one level past the first level that passes
    "jump_overshoot": ("    return lo;\n}\n\nint orc_insert(", "    return lo + 1;\n}\n\nint orc_insert("),
    # jump mode: the other movers counted on their level l as if they were above it
    "jump_counts_comovers": ("c += h->level[h->nbr[v][j]] >= x;", "c += h->level[h->nbr[v][j]] >= x - 1;"),
    # levels per group 4t replaced by t
    "group_size": ("T->Lg = lg_override > 0 ? lg_override : 4 * (t > 1 ? t : 1);",
                   "T->Lg = lg_override > 0 ? lg_override : (t > 1 ? t : 1);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = open(SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-shared", "-fPIC", "-w", "-o", str(so), str(mut)])
    env = dict(os.environ, PLDS_ORACLE_SO=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider",
                        "--deselect", "tests/test_oracle_pins.py::test_small_config_invariants_and_bound_every_batch"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
