"""Oracle for the hub-and-spoke matrix reordering (Algorithm 2, Section 3.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The bipartite network of Definition 1 has one instance node per row of A and
one feature node per column; every nonzero a_ij is an edge (i, j).  Global
node ids used for labels: instance i -> i, feature j -> m + j.

One iteration of Algorithm 2 on the active graph G = (I, F, E):
  1. m_hub = ceil(k * |I|), n_hub = ceil(k * |F|)          (hub selection)
     evaluated as an IEEE double product followed by ceil.
  2. deg(v) = number of edges from v to active nodes (degree in current G).
  3. hubs: active instances sorted by (deg desc, id asc), the first m_hub;
     same for features.  They are placed at the END of the order arrays, in
     sorted order filling inward, so the first (highest-degree) hub receives
     the highest new id (the Figure 2 caption: the hub instance gets id 9 of 9
     and the hub feature id 7 of 7).
  4. G' = G minus hubs.  Connected components of G' (isolated nodes are
     singleton components); the label of a component is its minimum global id.
  5. GCC = the component with the most nodes (instances + features), ties to
     the smallest label.
  6. every non-giant component, in ascending label order, takes the next
     free ids at the FRONT: its instances in ascending original id, its
     features likewise; each such component is one diagonal block of A11
     (possibly m_1i x 0 or 0 x n_1i).
  7. G <- GCC.  Stop when |I_GCC| < m_hub or |F_GCC| < n_hub (this
     iteration's hub counts), or when the GCC is empty.
After the loop the final GCC's nodes (ascending ids) fill the middle ids and
form the last diagonal block of A11.  Hubs form the trailing m2 rows / n2
columns; the spokes and the final GCC the leading m1 rows / n1 columns.

Readings where the paper is silent (tie-breaks, degree basis, placement of
the final GCC) are the ones listed above; the CUDA library implements the
same readings.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

__all__ = ["Reordering", "reorder", "hub_counts"]


@dataclasses.dataclass
class Reordering:
    m: int
    n: int
    row_order: np.ndarray   # new row position -> original row   (int64[m])
    col_order: np.ndarray   # new col position -> original col   (int64[n])
    row_off: np.ndarray     # block b holds new rows [row_off[b], row_off[b+1])
    col_off: np.ndarray     # and new cols [col_off[b], col_off[b+1])
    m1: int
    n1: int
    iterations: int
    hub_history: list       # per iteration (m_hub, n_hub, |I|, |F|)

    @property
    def m2(self) -> int:
        return self.m - self.m1

    @property
    def n2(self) -> int:
        return self.n - self.n1

    @property
    def num_blocks(self) -> int:
        return len(self.row_off) - 1

    @property
    def row_pos(self) -> np.ndarray:
        """pi_T of the paper: original row -> new position."""
        p = np.empty(self.m, dtype=np.int64)
        p[self.row_order] = np.arange(self.m)
        return p

    @property
    def col_pos(self) -> np.ndarray:
        """pi_F of the paper: original column -> new position."""
        p = np.empty(self.n, dtype=np.int64)
        p[self.col_order] = np.arange(self.n)
        return p


def hub_counts(k: float, n_inst: int, n_feat: int):
    """Hub counts of Algorithm 2 (hub selection step): ceil(k*|V_T|), ceil(k*|V_F|)."""
    return int(math.ceil(k * float(n_inst))), int(math.ceil(k * float(n_feat)))


def reorder(m: int, n: int, rowptr, col, k: float) -> Reordering:
    """Algorithm 2 on the bipartite network of A (CSR rowptr/col)."""
    if not (0.0 < k < 1.0):
        raise ValueError("hub ratio k must lie in (0, 1)")
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rowptr))
    cols = col

    act_T = np.ones(m, dtype=bool)
    act_F = np.ones(n, dtype=bool)
    row_order = np.full(m, -1, dtype=np.int64)
    col_order = np.full(n, -1, dtype=np.int64)
    fT, fF, bT, bF = 0, 0, m, n
    row_off = [0]
    col_off = [0]
    history = []
    it = 0
    gid_all = np.arange(m + n, dtype=np.int64)

    while True:
        nI = int(act_T.sum())
        nF = int(act_F.sum())
        if nI + nF == 0:
            break
        it += 1
        m_hub, n_hub = hub_counts(k, nI, nF)
        history.append((m_hub, n_hub, nI, nF))

        # degree of each active node in the current graph G
        e_act = act_T[rows] & act_F[cols]
        degT = np.bincount(rows[e_act], minlength=m)
        degF = np.bincount(cols[e_act], minlength=n)

        # hub selection: (deg desc, id asc); first hub gets the highest new id
        ids_T = np.nonzero(act_T)[0]
        ids_F = np.nonzero(act_F)[0]
        hubs_T = ids_T[np.lexsort((ids_T, -degT[ids_T]))][:m_hub]
        hubs_F = ids_F[np.lexsort((ids_F, -degF[ids_F]))][:n_hub]
        for h in hubs_T:
            bT -= 1
            row_order[bT] = h
        for h in hubs_F:
            bF -= 1
            col_order[bF] = h
        act_T[hubs_T] = False
        act_F[hubs_F] = False

        # connected components of G' (hubs removed); label = min global id
        e2 = act_T[rows] & act_F[cols]
        er, ec = rows[e2], cols[e2] + m
        g = sp.coo_matrix((np.ones(er.size, dtype=np.int8), (er, ec)), shape=(m + n, m + n)).tocsr()
        _, comp = connected_components(g, directed=False)
        active = np.concatenate([act_T, act_F])
        act_ids = gid_all[active]
        if act_ids.size == 0:
            break
        minid = np.full(comp.max() + 1, np.iinfo(np.int64).max, dtype=np.int64)
        np.minimum.at(minid, comp[act_ids], act_ids)
        label = np.full(m + n, -1, dtype=np.int64)
        label[act_ids] = minid[comp[act_ids]]

        # GCC = most nodes, ties to the smallest label
        labs, counts = np.unique(label[act_ids], return_counts=True)   # labs ascending
        best = np.lexsort((labs, -counts))[0]
        gcc = labs[best]

        # non-giant components take the next ids at the front, label ascending
        lab_T = label[:m]
        lab_F = label[m:]
        sel_T = np.nonzero(act_T & (lab_T != gcc))[0]
        sel_F = np.nonzero(act_F & (lab_F != gcc))[0]
        sel_T = sel_T[np.lexsort((sel_T, lab_T[sel_T]))]
        sel_F = sel_F[np.lexsort((sel_F, lab_F[sel_F]))]
        row_order[fT:fT + sel_T.size] = sel_T
        col_order[fF:fF + sel_F.size] = sel_F
        # block list in ascending label order
        ng = labs[labs != gcc]
        cT = np.searchsorted(ng, lab_T[sel_T])
        cF = np.searchsorted(ng, lab_F[sel_F])
        nT = np.bincount(cT, minlength=ng.size)
        nF_ = np.bincount(cF, minlength=ng.size)
        row_off.extend((fT + np.cumsum(nT)).tolist())
        col_off.extend((fF + np.cumsum(nF_)).tolist())
        fT += sel_T.size
        fF += sel_F.size

        # recurse on the GCC
        act_T &= (lab_T == gcc)
        act_F &= (lab_F == gcc)
        gI = int(act_T.sum())
        gF = int(act_F.sum())
        if gI < m_hub or gF < n_hub:
            break

    # the final GCC fills the middle ids and forms the last block of A11
    rest_T = np.nonzero(act_T)[0]
    rest_F = np.nonzero(act_F)[0]
    if rest_T.size + rest_F.size > 0:
        row_order[fT:fT + rest_T.size] = rest_T
        col_order[fF:fF + rest_F.size] = rest_F
        fT += rest_T.size
        fF += rest_F.size
        row_off.append(fT)
        col_off.append(fF)
    assert fT == bT and fF == bF, "front and back cursors must meet"
    return Reordering(m, n, row_order, col_order, np.asarray(row_off, dtype=np.int64),
                      np.asarray(col_off, dtype=np.int64), fT, fF, it, history)
