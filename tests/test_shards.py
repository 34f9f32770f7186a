"""Row-sharded build (Sec. 2 and 4.1: the matrix is split into row chunks of
about equal nonzero counts, one per process), host side on CPU.

- the shard boundaries of cih_shard_rows: monotone, covering 0 .. dim, each
  shard within one row of its equal share of the nonzeros;
- two gloo ranks (world_size 2) each take bench.py's rows for their rank,
  build them (here with the oracle: no GPU), and the gathered shards
  concatenate to the oracle's whole half-stored matrix; the job rate counts
  the matrix once and takes the slowest rank's time.
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cih():
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.mark.parametrize("sp,n", [((3, 3, 2, 0), 1), ((3, 3, 2, 0), 2), ((2, 2, 2, 0), 3), ((3, 3, 3, 1), 8),
                                  ((2, 1, 3, 1), 5)])
def test_shard_bounds_balance_the_nonzeros(cih, sp, n):
    S = oracle.Space(*sp)
    cnt = S.count_rows()
    rp = np.concatenate([[0], np.cumsum(cnt)])
    b = cih.shard_bounds(rp, n)
    assert b[0] == 0 and b[-1] == S.dim and np.all(np.diff(b) >= 0)
    nnz = rp[-1]
    for k in range(1, n):
        # shard k starts at the first row whose elements begin at or after k/n of the nonzeros
        assert rp[b[k]] >= nnz * k // n
        assert b[k] == 0 or rp[b[k] - 1] < nnz * k // n
    with pytest.raises(cih.CihError):
        cih.shard_bounds(rp, 0)


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sp = (3, 3, 2, 0)
        S = oracle.Space(*sp)
        t = synth.tbme_table(S.tbme_len, 4)
        rp = np.concatenate([[0], np.cumsum(S.count_rows())])
        r0, r1, nnz_s = bench.rank_rows(rp, world, rank)
        cnt, off, col, val = S.rows(np.arange(r0, r1, dtype=np.int64), t)
        assert int(cnt.sum()) == nnz_s
        shards = [None] * world
        dist.all_gather_object(shards, (r0, r1, col.tolist(), val.tolist()))
        ms = 10.0 + 5.0 * rank
        t_max = bench.max_over_ranks(ms, world, "cpu")
        out.put((rank, shards, t_max, bench.sharded_rate(3, int(rp[-1]), t_max)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_build_the_whole_matrix():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    S = oracle.Space(3, 3, 2, 0)
    rp_o, col_o, val_o = S.half_csr(synth.tbme_table(S.tbme_len, 4))
    for rank, shards, t_max, rate in res:
        assert [s[0] for s in shards] == [0, shards[0][1]] and shards[1][1] == S.dim
        col = np.concatenate([np.asarray(s[2], np.int32) for s in shards])
        val = np.concatenate([np.asarray(s[3], np.float32) for s in shards])
        np.testing.assert_array_equal(col, col_o)
        np.testing.assert_array_equal(val, val_o)
        assert t_max == 15.0
        assert rate == pytest.approx(3 * rp_o[-1] / 0.015)
