"""Louvain+ supergraph hierarchy, plain CPU oracle. TEST INFRASTRUCTURE ONLY.

Who may use this module: the tests, the smoke check in __graft_entry__ and the
CPU-baseline leg of bench.py. The product (the C-ABI library and its Python
binding) never imports or runs it and shares no code with it.

It follows the preprocessing step of Sec. 5 (the supergraph hierarchy, at most
k children per supernode and at most k supernodes at the top) and the
Louvain+ merge rules of Appendix A (Algorithmic Details): a level-(l+1)
supernode S is merged into a neighbouring supernode T either (i) when T is
S's only neighbour, or (ii) when T gives the largest modularity gain
Q^(S, T) = sum_{V_i in S} q(V_i, T). Every gain is an exact rational number
(fractions.Fraction), computed from the paper's q(V_i, T) formula term by
term, so no decision depends on rounding.

Readings where the appendix is silent (each also listed in the design notes):
  * the schedule: merges are decided in synchronous rounds. In a round every
    supernode S picks its target from the state at the start of the round;
    S moves when its target T does not move (T proposes nothing, or T
    proposes S back and T has the smaller id). A target takes its movers in
    increasing id order while the size cap holds; the others wait for a
    later round;
  * the size cap "less than k" of rule (ii) and the "at most k children" of
    Sec. 2.2 are read as: the merged supernode has at most k children, for
    rules (i) and (ii) alike;
  * rule (ii) first merges only on a positive gain (Louvain's merges); once
    a round of a level merges nothing, later rounds of that level also take
    the best non-positive gain, so that each level shrinks as far as the
    cap allows (Louvain+'s fix for Louvain's crowded top level);
  * a level ends with a round that merges nothing; the hierarchy ends when a
    level has at most k supernodes or merged nothing (a graph of more than k
    connected components keeps more than k supernodes at the top);
  * supernodes of a new level are numbered by their smallest child;
  * edges: the leaf CSR as given (both directions of an undirected edge),
    weights ignored, and 2m = the number of CSR entries. w(T) and
    w_cr(V_i, T) count ordered leaf pairs, i.e. both directions of each edge
    (w_cr: the entries u -> v and v -> u with u a leaf of V_i and v a leaf
    of T); w_in(.) is the degree sum. Only under this count is q(V_i, T)
    the change of modularity that the appendix calls it (it is then the
    move gain of Blondel et al.); with w_cr counting each crossing edge once
    its first term would be half the true one.

Parity status: pinned in tests/test_oracle_pins.py by the modularity of
Newman's definition (the gain of every merge equals the change of the
partition's modularity, brute force), the textbook split of two cliques
joined by a bridge, rule (i) on stars and paths, and the structural
invariants of the result.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

__all__ = ["louvain_plus", "louvain_gain", "modularity", "louvain_leaf_groups"]


def modularity(row_ptr, col, part) -> Fraction:
    """Newman's modularity of a partition of the leaves (exact):
    Q = sum_c [ e_c / m - (d_c / 2m)^2 ], e_c the undirected edges inside
    community c and d_c the sum of its leaves' degrees, with 2m = the number
    of CSR entries (both directions of each edge)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = len(row_ptr) - 1
    two_m = int(row_ptr[-1])
    inside, deg = {}, {}
    for u in range(n):
        cu = int(part[u])
        deg[cu] = deg.get(cu, 0) + int(row_ptr[u + 1] - row_ptr[u])
        for e in range(row_ptr[u], row_ptr[u + 1]):
            if int(part[int(col[e])]) == cu:
                inside[cu] = inside.get(cu, 0) + 1  # each inside edge twice
    q = Fraction(0)
    for c in deg:
        q += Fraction(inside.get(c, 0), two_m) - Fraction(deg[c], two_m) ** 2
    return q


def louvain_gain(children_S, T_children, leaves_of, row_ptr, col, level_of_leaf) -> Fraction:
    """Q^(S, T) of Appendix A: sum over the children V_i of S of
    q(V_i, T) = [(w(T) + w_cr(V_i, T)) / 2m - ((w_in(T) + w_in(V_i)) / 2m)^2]
              - [w(T) / 2m - (w_in(T) / 2m)^2 - (w_in(V_i) / 2m)^2],
    w(T) the leaf edges inside T, w_cr(V_i, T) the leaf edges between V_i and
    T (both as ordered pairs: each edge in both directions), w_in(.) the leaf
    edges incident to a supernode (its degree sum).
    `level_of_leaf[u]` is u's current level node; T_children is a set."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    two_m = Fraction(int(row_ptr[-1]))
    T_leaves = [u for A in sorted(T_children) for u in leaves_of[A]]
    w_T = 0  # ordered leaf pairs inside T (CSR entries: each inside edge twice)
    w_in_T = 0
    for u in T_leaves:
        w_in_T += int(row_ptr[u + 1] - row_ptr[u])
        for e in range(row_ptr[u], row_ptr[u + 1]):
            if level_of_leaf[int(col[e])] in T_children:
                w_T += 1
    total = Fraction(0)
    for Vi in sorted(children_S):
        w_in_i = 0
        w_cr = 0  # ordered leaf pairs between V_i and T: both directions
        for u in leaves_of[Vi]:
            w_in_i += int(row_ptr[u + 1] - row_ptr[u])
            for e in range(row_ptr[u], row_ptr[u + 1]):
                if level_of_leaf[int(col[e])] in T_children:
                    w_cr += 2  # u -> v here, v -> u in v's row
        a = (w_T + w_cr) / two_m - ((w_in_T + w_in_i) / two_m) ** 2
        b = w_T / two_m - (w_in_T / two_m) ** 2 - (w_in_i / two_m) ** 2
        total += a - b
    return total


def _one_level(n_level, leaves_of, row_ptr, col, level_of_leaf, k):
    """Groups the n_level nodes of one level into the next level's supernodes
    (the synchronous rounds of the readings above). Returns the parent of
    every node of this level, numbered by smallest child."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    children = {A: {A} for A in range(n_level)}  # group id -> its nodes of this level
    group_of = list(range(n_level))
    relaxed = False
    while True:
        # state at the start of the round
        leaf_group = [group_of[level_of_leaf[u]] for u in range(len(row_ptr) - 1)]
        neighbours = {S: set() for S in children}
        for u in range(len(row_ptr) - 1):
            for e in range(row_ptr[u], row_ptr[u + 1]):
                S, T = leaf_group[u], leaf_group[int(col[e])]
                if S != T:
                    neighbours[S].add(T)
        prop = {}
        for S in sorted(children):
            fits = [T for T in sorted(neighbours[S]) if len(children[S]) + len(children[T]) <= k]
            if not fits:
                continue
            if len(neighbours[S]) == 1:  # rule (i): T is S's only neighbour
                prop[S] = fits[0]
                continue
            best, best_T = None, None
            for T in fits:  # rule (ii): the largest gain, ties to the smaller id
                gain = louvain_gain(children[S], children[T], leaves_of, row_ptr, col, level_of_leaf)
                if best is None or gain > best:
                    best, best_T = gain, T
            if relaxed or best > 0:
                prop[S] = best_T
        movers = {}
        for S, T in prop.items():
            if T not in prop or (prop[T] == S and S > T):
                movers.setdefault(T, []).append(S)
        accepted = []
        for T in sorted(movers):
            room = k - len(children[T])
            for S in sorted(movers[T]):
                if len(children[S]) <= room:
                    accepted.append((S, T))
                    room -= len(children[S])
        if not accepted:
            if relaxed:
                break
            relaxed = True
            continue
        for S, T in accepted:
            children[T] |= children.pop(S)
            for A in children[T]:
                group_of[A] = T
    firsts = sorted(min(c) for c in children.values())
    new_id = {first: i for i, first in enumerate(firsts)}
    return [new_id[min(children[group_of[A]])] for A in range(n_level)]


def louvain_plus(n, row_ptr, col, k):
    """The Louvain+ hierarchy of Sec. 5 / Appendix A on an undirected CSR.
    Returns [p_1, p_2, ...]: p_l[A] is the level-l supernode of level-(l-1)
    node A (level 0 = the leaves). Empty when n <= k or nothing merges."""
    if k < 2:
        raise ValueError("Louvain+ needs k >= 2")
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    level_of_leaf = list(range(n))
    n_level = n
    leaves_of = {A: [A] for A in range(n)}
    levels = []
    while n_level > k:
        parent = _one_level(n_level, leaves_of, row_ptr, col, level_of_leaf, k)
        n_next = max(parent) + 1 if parent else 0
        if n_next == n_level:
            break
        levels.append(np.asarray(parent, dtype=np.int64))
        level_of_leaf = [parent[level_of_leaf[u]] for u in range(n)]
        leaves_of = {}
        for u in range(n):
            leaves_of.setdefault(level_of_leaf[u], []).append(u)
        n_level = n_next
    return levels


def louvain_leaf_groups(n, levels):
    """The level-l supernode of every leaf, for l = 1..L (composes the
    parent arrays)."""
    out = []
    cur = np.arange(n, dtype=np.int64)
    for p in levels:
        cur = np.asarray(p, dtype=np.int64)[cur]
        out.append(cur.copy())
    return out
