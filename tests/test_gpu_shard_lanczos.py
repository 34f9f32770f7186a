"""Lanczos over row shards (cih_lanczos_lowest_shard, cih_ham_upper_sumsq):
the matrix split over processes in chunks of equal nonzero count, as the
paper distributes it (Sec. 2 and 4.1).  Each product runs on the local rows;
a caller callback sums the row part (FP64, one nonzero term per entry) and
the fixed-point mirror accumulators (integers) over the processes, both
exactly, so every process follows the same Lanczos run as one process on the
whole matrix.

The two-process test runs two gloo ranks on the one GPU: their kernels never
wait on each other (the sums go through host copies between launches).
"""
import os

import numpy as np
import pytest

from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
SP = (3, 3, 4, 0)


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.mark.parametrize("K", [1, 3])
def test_one_shard_equals_the_whole_run(cih, K):
    """One process holding every row, with a combine that has nothing to add:
    the same bits as cih_lanczos_lowest."""
    B = cih.Basis(*SP)
    T = torch.from_numpy(synth.tbme_tables(B.tbme_len, list(range(7, 7 + K)))).cuda()
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, T)
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=300, tol=1e-10)
    calls = []
    f2 = B.upper_sumsq(rowptr, 0, B.dim, val)
    ev_s, psi_s, conv_s = B.lanczos_shard(rowptr, 0, B.dim, col, val, f2, lambda a, y: calls.append(1),
                                          nev=5, max_iter=300, tol=1e-10)
    assert conv and conv_s and len(calls) > 5
    np.testing.assert_array_equal(ev_s, ev)
    assert torch.equal(psi_s, psi)


def test_shard_arguments(cih):
    B = cih.Basis(*SP)
    rowptr, nnz = B.count()
    with pytest.raises(cih.CihError):
        B.upper_sumsq(rowptr, 5, 2, torch.zeros((1, 0), device="cuda"))
    assert B.upper_sumsq(rowptr, 3, 3, torch.zeros((1, 0), device="cuda")) == 0.0

    def bad(a, y):
        raise RuntimeError("combine failed")
    col, val = B.fill(rowptr, nnz, torch.from_numpy(synth.tbme_table(B.tbme_len, 1)).cuda())
    with pytest.raises(RuntimeError):
        B.lanczos_shard(rowptr, 0, B.dim, col, val, 1.0, bad, nev=1, max_iter=20, tol=1e-8)


def _rank_main(rank, world, port, K, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1412_5989_gb300 import cih
        torch.cuda.set_device(0)
        B = cih.Basis(*SP)
        T = torch.from_numpy(synth.tbme_tables(B.tbme_len, list(range(7, 7 + K)))).cuda()
        rowptr, nnz = B.count()
        b = cih.shard_bounds(rowptr.cpu().numpy(), world)
        r0, r1 = int(b[rank]), int(b[rank + 1])
        col, val = B.fill_rows(rowptr, r0, r1, T)
        ev, psi, conv = cih.lanczos_distributed(B, rowptr, r0, r1, col, val, nev=5, max_iter=300, tol=1e-10)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), ev=ev, psi=psi.cpu().numpy(), conv=conv, r0=r0, r1=r1)
        B.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("K", [1, 2])
def test_two_processes_follow_the_whole_run(cih, K, tmp_path):
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, K, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    assert res[0]["r0"] == 0 and res[0]["r1"] == res[1]["r0"] and res[0]["r1"] > 0
    np.testing.assert_array_equal(res[0]["ev"], res[1]["ev"])            # every process, the same run
    np.testing.assert_array_equal(res[0]["psi"], res[1]["psi"])
    assert bool(res[0]["conv"])
    B = cih.Basis(*SP)
    T = torch.from_numpy(synth.tbme_tables(B.tbme_len, list(range(7, 7 + K)))).cuda()
    rowptr, col, val, nnz = cih.build_hamiltonian(B, T)
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=300, tol=1e-10)
    assert res[1]["r1"] == B.dim
    # the same run as one process, unless the summed bound lands on the other
    # side of a power of two (then the mirrored part's units differ by 2)
    np.testing.assert_allclose(res[0]["ev"], ev, rtol=1e-12, atol=0)
