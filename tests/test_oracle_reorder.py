"""Pins for the reordering oracle (Algorithm 2, Section 3.2).

The oracle is checked against (a) hand-derived golden cases, one built from
the facts of the Figure 2 caption, (b) invariants that any correct result of
Algorithm 2 satisfies whatever the implementation (a permutation; A11 block
diagonal over the emitted blocks; every block a connected component; hub
counts ceil(k |V|); the first hubs are the top-degree nodes of A), and (c) a
brute-force pure-Python BFS re-run on tiny random graphs.
"""
import json
import math
import os
from collections import deque

import numpy as np
import pytest

from oracle.reorder import reorder, hub_counts
import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _csr_from_edges(m, n, edges):
    edges = sorted(set(map(tuple, edges)))
    rowptr = np.zeros(m + 1, dtype=np.int64)
    for r, _ in edges:
        rowptr[r + 1] += 1
    rowptr = np.cumsum(rowptr)
    col = np.array([c for _, c in edges], dtype=np.int32)
    return rowptr, col


@pytest.mark.parametrize("name", ["fig2_toy.json", "star.json", "one_side_stop.json"])
def test_golden_hand_derived(name):
    g = json.load(open(os.path.join(GOLD, name)))
    rowptr, col = _csr_from_edges(g["m"], g["n"], g["edges_row_col"])
    R = reorder(g["m"], g["n"], rowptr, col, g["k"])
    assert R.row_order.tolist() == g["row_order"]
    assert R.col_order.tolist() == g["col_order"]
    assert R.row_off.tolist() == g["row_off"]
    assert R.col_off.tolist() == g["col_off"]
    assert (R.m1, R.n1, R.iterations) == (g["m1"], g["n1"], g["iterations"])


def test_fig2_caption_facts():
    """Figure 2 caption: hub instance -> id 9, hub feature -> id 7, spokes lowest ids."""
    g = json.load(open(os.path.join(GOLD, "fig2_toy.json")))
    rowptr, col = _csr_from_edges(g["m"], g["n"], g["edges_row_col"])
    R = reorder(g["m"], g["n"], rowptr, col, g["k"])
    pos_T, pos_F = R.row_pos, R.col_pos
    assert pos_T[8] + 1 == 9 and pos_F[6] + 1 == 7
    assert sorted((pos_T[[0, 1, 2]] + 1).tolist()) == [1, 2, 3] and pos_F[0] + 1 == 1


def _bfs_components(nodes, adj):
    seen, comps = set(), []
    for s in sorted(nodes):
        if s in seen:
            continue
        comp, dq = [], deque([s])
        seen.add(s)
        while dq:
            u = dq.popleft()
            comp.append(u)
            for v in adj[u]:
                if v in nodes and v not in seen:
                    seen.add(v)
                    dq.append(v)
        comps.append(sorted(comp))
    return comps


def _brute_reorder(m, n, edges, k):
    """Algorithm 2 with explicit loops and BFS (independent of the vectorised oracle)."""
    adj = {v: set() for v in range(m + n)}
    for r, c in edges:
        adj[r].add(m + c)
        adj[m + c].add(r)
    I, F = set(range(m)), set(range(m, m + n))
    front_T, front_F, back_T, back_F = [], [], [], []
    while I or F:
        mh = math.ceil(k * len(I))
        nh = math.ceil(k * len(F))
        act = I | F
        deg = {v: len(adj[v] & act) for v in act}
        hT = sorted(I, key=lambda v: (-deg[v], v))[:mh]
        hF = sorted(F, key=lambda v: (-deg[v], v))[:nh]
        back_T += hT
        back_F += [v - m for v in hF]
        I -= set(hT)
        F -= set(hF)
        comps = _bfs_components(I | F, adj)
        if not comps:
            break
        gcc = sorted(comps, key=lambda c: (-len(c), c[0]))[0]
        for c in sorted(comps, key=lambda c: c[0]):
            if c is gcc:
                continue
            front_T += [v for v in c if v < m]
            front_F += [v - m for v in c if v >= m]
        I = {v for v in gcc if v < m}
        F = {v for v in gcc if v >= m}
        if len(I) < mh or len(F) < nh:
            break
    front_T += sorted(I)
    front_F += sorted(v - m for v in F)
    return front_T + back_T[::-1], front_F + back_F[::-1]


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(3, 13)), int(rng.integers(2, 10))
    dens = rng.uniform(0.1, 0.5)
    rowptr, col, _ = workloads.make_tiny_random(m, n, dens, rng)
    k = float(rng.choice([0.05, 0.1, 0.2, 0.34]))
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    edges = list(zip(rows.tolist(), col.tolist()))
    R = reorder(m, n, rowptr, col, k)
    bt, bf = _brute_reorder(m, n, edges, k)
    assert R.row_order.tolist() == bt
    assert R.col_order.tolist() == bf


def _check_invariants(m, n, rowptr, col, k, R):
    assert sorted(R.row_order.tolist()) == list(range(m))
    assert sorted(R.col_order.tolist()) == list(range(n))
    pT, pF = R.row_pos, R.col_pos
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    nr, nc = pT[rows], pF[np.asarray(col)]
    # A11 is block diagonal over the emitted blocks
    ro, co = R.row_off, R.col_off
    assert ro[0] == 0 and co[0] == 0 and ro[-1] == R.m1 and co[-1] == R.n1
    assert np.all(np.diff(ro) >= 0) and np.all(np.diff(co) >= 0)
    in11 = (nr < R.m1) & (nc < R.n1)
    rb = np.searchsorted(ro, nr[in11], side="right") - 1
    cb = np.searchsorted(co, nc[in11], side="right") - 1
    assert np.array_equal(rb, cb)
    # every block is connected inside A11 (a single component)
    B = len(ro) - 1
    adj = {}
    for a, b in zip(nr[in11].tolist(), nc[in11].tolist()):
        adj.setdefault(("r", a), set()).add(("c", b))
        adj.setdefault(("c", b), set()).add(("r", a))
    for b in range(B):
        nodes = [("r", i) for i in range(ro[b], ro[b + 1])] + [("c", j) for j in range(co[b], co[b + 1])]
        assert len(nodes) >= 1
        seen, dq = {nodes[0]}, deque([nodes[0]])
        while dq:
            u = dq.popleft()
            for v in adj.get(u, ()):
                if v not in seen:
                    seen.add(v)
                    dq.append(v)
        assert seen == set(nodes), f"block {b} is not connected"
    # hub counts are ceil(k |V|) of each iteration and their sum is m2 / n2
    assert sum(h[0] for h in R.hub_history) == R.m2
    assert sum(h[1] for h in R.hub_history) == R.n2
    for mh, nh, nI, nF in R.hub_history:
        assert (mh, nh) == hub_counts(k, nI, nF)
    # the first iteration's hubs are the top-degree rows/cols of A (deg desc, id asc)
    mh, nh = R.hub_history[0][:2]
    degT = np.diff(rowptr)
    degF = np.bincount(np.asarray(col), minlength=n)
    topT = sorted(range(m), key=lambda v: (-degT[v], v))[:mh]
    topF = sorted(range(n), key=lambda v: (-degF[v], v))[:nh]
    assert R.row_order[m - mh:][::-1].tolist() == topT
    assert R.col_order[n - nh:][::-1].tolist() == topF


@pytest.mark.parametrize("seed", range(6))
def test_invariants_random_powerlaw(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 300, 80
    rowptr, col, _ = workloads.chung_lu_csr(m, n, 900, 2.1, rng)
    k = [0.01, 0.02, 0.05, 0.1, 0.2, 0.5][seed]
    R = reorder(m, n, rowptr, col, k)
    _check_invariants(m, n, rowptr, col, k, R)


def test_invariants_small_workload():
    w = workloads.make("small", with_y=False)
    R = reorder(w["m"], w["n"], w["rowptr"], w["col"], w["cfg"].k)
    _check_invariants(w["m"], w["n"], w["rowptr"], w["col"], w["cfg"].k, R)


def test_disjoint_blocks_plus_global_hub():
    """Three dense 2x2 blocks plus one instance and one feature touching everything.

    Hand derivation (k = 0.1, one hub per side per iteration):
    it1 removes instance 6 and feature 6 (degree 7); the three 2x2 blocks are
    the components, the first (label 0) is the GCC by the smallest-label tie,
    the other two become the A11 blocks in label order.  it2 takes instance 0
    and feature 0 (degree 2, lowest id) from the GCC, leaving {i1, f1} as the
    new GCC; it3 takes those as hubs and the graph is empty."""
    m, n = 7, 7
    edges = []
    for b in range(3):
        for i in range(2):
            for j in range(2):
                edges.append((2 * b + i, 2 * b + j))
    edges += [(6, j) for j in range(7)] + [(i, 6) for i in range(7)]
    rowptr, col = _csr_from_edges(m, n, edges)
    R = reorder(m, n, rowptr, col, 0.1)
    assert R.row_order.tolist() == [2, 3, 4, 5, 1, 0, 6]
    assert R.col_order.tolist() == [2, 3, 4, 5, 1, 0, 6]
    assert R.row_off.tolist() == [0, 2, 4] and R.col_off.tolist() == [0, 2, 4]
    assert (R.m1, R.n1, R.iterations) == (4, 4, 3)


def test_empty_rows_and_columns():
    """Rows / columns with no nonzero are isolated nodes: singleton components."""
    m, n = 6, 5
    edges = [(0, 0), (1, 0), (1, 1), (2, 1), (3, 3)]
    rowptr, col = _csr_from_edges(m, n, edges)
    R = reorder(m, n, rowptr, col, 0.2)
    _check_invariants(m, n, rowptr, col, 0.2, R)
    bt, bf = _brute_reorder(m, n, edges, 0.2)
    assert R.row_order.tolist() == bt and R.col_order.tolist() == bf


def test_path_graph():
    m, n = 8, 7
    edges = [(i, i) for i in range(7)] + [(i + 1, i) for i in range(7)]
    rowptr, col = _csr_from_edges(m, n, edges)
    R = reorder(m, n, rowptr, col, 0.1)
    _check_invariants(m, n, rowptr, col, 0.1, R)
    bt, bf = _brute_reorder(m, n, edges, 0.1)
    assert R.row_order.tolist() == bt and R.col_order.tolist() == bf


def test_rejects_bad_k():
    with pytest.raises(ValueError):
        reorder(2, 2, np.array([0, 1, 2]), np.array([0, 1]), 1.0)
