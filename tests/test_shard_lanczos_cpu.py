"""CPU, two gloo ranks: the cross-process part of the Lanczos over row shards
(cih.lanczos_distributed).  A stand-in for the basis records what the library
would receive: the bound each rank passes (the sum of the shards'
upper_sumsq over the ranks) and the two product buffers after the combine
callback (the sum over the ranks: integer accumulators, and FP64 row parts
with one nonzero term per entry).  The GPU side of the same path runs in
tests/test_gpu_shard_lanczos.py."""
import os

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


class _StandInBasis:
    """upper_sumsq / lanczos_shard with the library's call signature; the
    "product" puts rank-dependent values in the two buffers and combines them
    twice, as two Lanczos steps would."""

    def __init__(self, rank, dim=6):
        self.rank, self.dim = rank, dim

    def upper_sumsq(self, rowptr, r0, r1, val, element_major=False):
        return 10.0 * (self.rank + 1) + 0.25

    def lanczos_shard(self, rowptr, r0, r1, col, val, f2, combine, nev, max_iter, tol, want_vectors, element_major):
        out = {"f2": f2, "steps": []}
        for step in range(2):
            acc = torch.zeros(self.dim, dtype=torch.int64)
            yx = torch.zeros(self.dim, dtype=torch.float64)
            acc[:] = (self.rank + 1) * (step + 1)
            acc[self.rank] = -(2 ** 62) + self.rank          # large integers sum exactly
            yx[self.rank * 3:(self.rank + 1) * 3] = 0.1 * (self.rank + 1) + step
            combine(acc, yx)
            out["steps"].append((acc.tolist(), yx.tolist()))
        return out, None, True


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1412_5989_gb300 import cih
        out, _, conv = cih.lanczos_distributed(_StandInBasis(rank), None, 3 * rank, 3 * rank + 3, None,
                                               torch.zeros((1, 1)))
        q.put((rank, out, conv))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_the_bound_and_the_buffers():
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
    for rank, out, conv in res:
        assert conv
        assert out["f2"] == (10.25 + 20.25)                          # the same bound on every rank
        for step, (acc, yx) in enumerate(out["steps"]):
            want_acc = [(1 + 2) * (step + 1)] * 6
            want_acc[0] = -(2 ** 62) + 0 + 2 * (step + 1)
            want_acc[1] = -(2 ** 62) + 1 + 1 * (step + 1)
            assert acc == want_acc
            assert yx == [0.1 + step] * 3 + [0.2 + step] * 3           # one nonzero term per entry
    assert res[0][1] == res[1][1]
