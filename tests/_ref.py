"""Pure-Python references for small graphs (test-only, slow on purpose).

- ``brute_coreness``: coreness(v) = max over vertex subsets S containing v of the
  minimum degree of the induced subgraph G[S] (definition of k-core / coreness,
  Section "Preliminaries").  Exponential; n <= 12.
- ``GlobalPLDS``: the batch rules written as a global fixpoint instead of the
  oracle's candidate bookkeeping.  Insertion (Algorithm 2): for l = 0..K-1 move
  *every* vertex on level l whose up-degree exceeds the level's cutoff.  Deletion
  (Algorithm 3): repeatedly take all vertices violating Invariant 2, compute their
  desire-levels from the Definition, and move those with the smallest one.  This
  checks the oracle's incremental candidate tracking on tiny graphs.
- ``fraction_tables``: thresholds with Python's ``fractions`` module.
"""
from __future__ import annotations

import math
from fractions import Fraction
from itertools import combinations


def rational(x: float) -> Fraction:
    return Fraction(round(x * 10**6), 10**6)


def fraction_tables(n, delta=0.4, lam=3.0, levels_per_group=0):
    d = rational(delta)
    lm = rational(lam)
    base = 1 + d
    t = 0
    while base ** t < n:
        t += 1
    Lg = levels_per_group or 4 * max(1, t)
    G = t + 1
    c = 2 + Fraction(3) / lm
    upmax = [min(math.floor(c * base ** i), n) for i in range(G)]
    dnmin = [min(math.ceil(base ** i), n) for i in range(G)]
    return dict(t=t, Lg=Lg, G=G, K=G * Lg, upmax=upmax, dnmin=dnmin)


def brute_coreness(n, edges):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[int(u)].add(int(v))
        adj[int(v)].add(int(u))
    core = [0] * n
    for mask in range(1, 1 << n):
        S = [v for v in range(n) if mask >> v & 1]
        mind = min(sum(1 for w in adj[v] if mask >> w & 1) for v in S)
        for v in S:
            if mind > core[v]:
                core[v] = mind
    return core


class GlobalPLDS:
    def __init__(self, n, delta=0.4, lam=3.0, levels_per_group=0):
        T = fraction_tables(n, delta, lam, levels_per_group)
        self.n, self.Lg, self.K = n, T["Lg"], T["K"]
        self.upmax, self.dnmin = T["upmax"], T["dnmin"]
        self.level = [0] * n
        self.adj = [set() for _ in range(n)]

    def gn(self, l):
        return l // self.Lg

    def cnt(self, v, x):
        return sum(1 for w in self.adj[v] if self.level[w] >= x)

    def up(self, v):
        return self.cnt(v, self.level[v])

    def upstar(self, v):
        return self.cnt(v, self.level[v] - 1)

    def _keys(self, edges):
        out = set()
        for u, v in edges:
            u, v = int(u), int(v)
            if u != v:
                out.add((min(u, v), max(u, v)))
        return sorted(out)

    def insert(self, edges):
        for u, v in self._keys(edges):
            self.adj[u].add(v)
            self.adj[v].add(u)
        for l in range(self.K):
            movers = [v for v in range(self.n)
                      if self.level[v] == l and self.up(v) > self.upmax[self.gn(l)]]
            for v in movers:
                self.level[v] = l + 1

    def _violates2(self, v):
        l = self.level[v]
        return l > 0 and self.upstar(v) < self.dnmin[self.gn(l - 1)]

    def _dl(self, v):
        for lp in range(self.level[v] - 1, -1, -1):
            ok2 = lp == 0 or self.cnt(v, lp - 1) >= self.dnmin[self.gn(lp - 1)]
            ok1 = self.cnt(v, lp) <= self.upmax[self.gn(lp)]
            if ok1 and ok2:
                return lp
        return 0

    def delete(self, edges):
        for u, v in self._keys(edges):
            self.adj[u].discard(v)
            self.adj[v].discard(u)
        while True:
            viol = [v for v in range(self.n) if self._violates2(v)]
            if not viol:
                break
            dls = {v: self._dl(v) for v in viol}
            lo = min(dls.values())
            for v, d in dls.items():
                if d == lo:
                    self.level[v] = lo


def within_bound(est_exponent, core, delta_num=2, delta_den=5, c_num=3, c_den=1):
    """Exact check of k/c' <= khat <= c' k with c' = (2+3/lambda)(1+delta).

    khat = (1+delta)^g; with 1+delta = a/b and c = (2+3/lambda) = p/q the bound
    c' = p a / (q b).  Returns False on any violation; khat=0 iff core=0.
    """
    a, b = delta_den + delta_num, delta_den
    for g, k in zip(est_exponent, core):
        g, k = int(g), int(k)
        if k == 0 or g < 0:
            if not (k == 0 and g < 0):
                return False
            continue
        khat = Fraction(a ** g, b ** g)
        cprime = Fraction(c_num * a, c_den * b)
        if not (Fraction(k) <= cprime * khat and khat <= cprime * k):
            return False
    return True


def all_pairs(n):
    return list(combinations(range(n), 2))
