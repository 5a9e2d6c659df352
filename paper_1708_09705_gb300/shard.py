"""Row-sharded split of one field's covariance over several GPUs (host-side
plan).

The hot path of one field has one exchange step: the products with B =
I + S^1/2 K S^1/2 need, on every rank, the entries of the multiplied vector
at the neighbours of its rows.  With the stars spatially sorted, a
contiguous block of rows is a compact sky tile, so each rank needs only the
vector entries of the stars within the cutoff of its tile's edge (its halo);
the CG scalars are sums over all rows (one all-reduce per dot product); the
EP site updates are local (Sect. 4.1: sites are exchanged once per EP
iteration, all per-star work is independent).

`plan_rows` cuts the rows into contiguous blocks of equal stored entries and
lists, per rank, the halo columns it receives and the rows it sends to each
peer.  `local_csr` renumbers a rank's rows into its [own rows | halo] vector
layout.  The single-GPU build runs neither: this module fixes the partition
and the exchange lists that a multi-GPU run would use, and the tests check
one sharded product and one all-reduced dot on CPU ranks against the
single-rank result.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class RankPlan:
    rank: int
    r0: int                      # first owned row
    r1: int                      # one past the last owned row
    halo: np.ndarray             # sorted global columns outside [r0, r1) that the rows use
    recv: dict = field(default_factory=dict)   # peer -> global rows received (sorted)
    send: dict = field(default_factory=dict)   # peer -> global rows sent (sorted, owned)


def plan_rows(row_ptr: np.ndarray, col: np.ndarray, world: int) -> list[RankPlan]:
    """Contiguous row blocks with (nearly) equal stored entries, and the
    halo exchange lists between them."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    if world < 1:
        raise ValueError("world must be >= 1")
    nnz = int(row_ptr[-1])
    # block boundaries: the first row whose prefix count reaches k * nnz / world
    cuts = [0]
    for k in range(1, world):
        cuts.append(int(np.searchsorted(row_ptr, k * nnz / world, side="left")))
    cuts.append(n)
    cuts = list(np.maximum.accumulate(np.minimum(cuts, n)))
    plans = []
    for r in range(world):
        r0, r1 = cuts[r], cuts[r + 1]
        cols = col[row_ptr[r0]:row_ptr[r1]]
        halo = np.unique(cols[(cols < r0) | (cols >= r1)])
        plans.append(RankPlan(r, r0, r1, halo))
    for p in plans:
        for q in plans:
            if p.rank == q.rank:
                continue
            need = p.halo[(p.halo >= q.r0) & (p.halo < q.r1)]
            if len(need):
                p.recv[q.rank] = need
                q.send[p.rank] = need
    return plans


def local_csr(row_ptr, col, val, p: RankPlan):
    """The rank's rows with columns renumbered into its vector layout
    [owned rows (r1 - r0 entries) | halo (len(p.halo) entries)]."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    lo, hi = row_ptr[p.r0], row_ptr[p.r1]
    c = np.asarray(col[lo:hi], dtype=np.int64)
    own = (c >= p.r0) & (c < p.r1)
    lc = np.empty_like(c)
    lc[own] = c[own] - p.r0
    lc[~own] = (p.r1 - p.r0) + np.searchsorted(p.halo, c[~own])
    return row_ptr[p.r0:p.r1 + 1] - lo, lc, np.asarray(val[lo:hi])
