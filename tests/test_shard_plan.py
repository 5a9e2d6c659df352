"""Row-sharded product of one field over CPU ranks (gloo): the partition and
halo lists of paper_1708_09705_gb300.shard, one product K x with a halo
exchange and one all-reduced dot, against the single-rank result."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1708_09705_gb300 import shard
from synth import catalogue_subset, make_catalogue


def _field(n=300):
    cat = catalogue_subset(make_catalogue("c1_plain_400", truth="mean"), np.arange(n))
    u = O.unit_vectors(cat["l"], cat["b"])
    x = u * cat["s"][:, None]
    # the library's internal order: sorted along the field (a spatial sort)
    order = np.lexsort((x[:, 2], x[:, 1], x[:, 0]))
    x = x[order]
    pairs = O.neighbour_pairs(x, float(cat["cutoff_pc"]))
    rp, col = O.csr_structure(n, pairs)
    rng = np.random.default_rng(1)
    w = rng.uniform(0.1, 1.0, len(pairs))
    vals = {(i, j): v for (i, j), v in zip(map(tuple, pairs), w)}
    val = np.array([1.0 if i == j else vals[(min(i, j), max(i, j))]
                    for i, j in zip(np.repeat(np.arange(n), np.diff(rp)), col)])
    return rp, col, val


def test_plan_covers_rows_and_balances_entries():
    rp, col, val = _field()
    n = len(rp) - 1
    for world in (1, 2, 3, 5):
        plans = shard.plan_rows(rp, col, world)
        assert plans[0].r0 == 0 and plans[-1].r1 == n
        assert all(plans[k].r1 == plans[k + 1].r0 for k in range(world - 1))
        counts = [rp[p.r1] - rp[p.r0] for p in plans]
        # each boundary is off its target by less than one row
        assert max(counts) - min(counts) <= 2 * np.diff(rp).max()
        for p in plans:
            # every column a rank's rows use is owned or in its halo
            cols = col[rp[p.r0]:rp[p.r1]]
            outside = cols[(cols < p.r0) | (cols >= p.r1)]
            assert set(outside.tolist()) == set(p.halo.tolist())
            # what a rank receives from q is exactly what q sends to it
            for q, rows in p.recv.items():
                np.testing.assert_array_equal(plans[q].send[p.rank], rows)
            got = np.concatenate([p.recv[q] for q in sorted(p.recv)]) if p.recv else []
            assert sorted(np.asarray(got).tolist()) == p.halo.tolist()


def _rank_main(rank, world, port, rp, col, val, xg, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plans = shard.plan_rows(rp, col, world)
        p = plans[rank]
        xl = torch.tensor(xg[p.r0:p.r1])
        # halo exchange: point-to-point sends of owned entries, receives of halo entries
        reqs, bufs = [], {}
        for q, rows in p.send.items():
            reqs.append(dist.isend(xl[torch.tensor(rows - p.r0)].contiguous(), q))
        for q, rows in p.recv.items():
            bufs[q] = torch.empty(len(rows), dtype=xl.dtype)
            reqs.append(dist.irecv(bufs[q], q))
        for r in reqs:
            r.wait()
        halo = torch.empty(len(p.halo), dtype=xl.dtype)
        for q, rows in p.recv.items():
            halo[torch.tensor(np.searchsorted(p.halo, rows))] = bufs[q]
        xv = torch.cat([xl, halo]).numpy()
        lrp, lcol, lval = shard.local_csr(rp, col, val, p)
        y = np.array([np.dot(lval[lrp[i]:lrp[i + 1]], xv[lcol[lrp[i]:lrp[i + 1]]])
                      for i in range(p.r1 - p.r0)])
        # one CG dot: local partial, all-reduced
        d = torch.tensor([float(np.dot(y, xg[p.r0:p.r1]))], dtype=torch.float64)
        dist.all_reduce(d)
        out.put((rank, p.r0, p.r1, y, float(d[0])))
    finally:
        dist.destroy_process_group()


def test_sharded_product_and_dot_match_single_rank():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    rp, col, val = _field()
    n = len(rp) - 1
    xg = np.random.default_rng(2).standard_normal(n)
    yref = np.array([np.dot(val[rp[i]:rp[i + 1]], xg[col[rp[i]:rp[i + 1]]]) for i in range(n)])
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, rp, col, val, xg, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    y = np.empty(n)
    dots = set()
    for rank, r0, r1, yl, d in res:
        y[r0:r1] = yl
        dots.add(d)
    np.testing.assert_allclose(y, yref, rtol=1e-13, atol=1e-13)
    assert len(dots) == 1
    assert dots.pop() == pytest.approx(float(np.dot(yref, xg)), rel=1e-12)
