"""GPU: the row-sharded fill (cih_ham_fill_rows) as logical shards on one GPU.

Shards of about equal nonzeros (cih_shard_rows), each filled into arrays
holding only its rows, concatenate to the whole fill bit for bit: one table
at 4+4 Nmax=4, two tables with a one-body override at 3+3 Nmax=4, and the
degenerate shards (empty ranges, a single row)."""
import numpy as np
import pytest

from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.mark.parametrize("sp,n,K,override", [((4, 4, 4, 0), 2, 1, False), ((4, 4, 4, 0), 3, 1, False),
                                             ((3, 3, 4, 0), 4, 2, True)])
def test_shards_concatenate_to_the_whole_fill(cih, sp, n, K, override):
    B = cih.Basis(*sp)
    T = torch.from_numpy(synth.tbme_tables(B.tbme_len, range(5, 5 + K))).cuda()
    esp = torch.from_numpy(synth.single_particle_energies(sum(B.n_orb), 6)) if override else None
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, T, e_sp=esp)
    bounds = cih.shard_bounds(rowptr.cpu().numpy(), n)
    parts = [B.fill_rows(rowptr, int(bounds[k]), int(bounds[k + 1]), T, e_sp=esp) for k in range(n)]
    B.check()
    assert torch.equal(torch.cat([p[0] for p in parts]), col)
    assert torch.equal(torch.cat([p[1] for p in parts], dim=1), val)
    sizes = [p[0].numel() for p in parts]
    assert max(sizes) - min(sizes) <= int((rowptr[1:] - rowptr[:-1]).max().item())   # balanced within a row


def test_degenerate_shards(cih):
    B = cih.Basis(3, 3, 2, 0)
    T = torch.from_numpy(synth.tbme_table(B.tbme_len, 1)).cuda()
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, T)
    rp = rowptr.cpu().numpy()
    c0, v0 = B.fill_rows(rowptr, 7, 7, T)                    # empty range: nothing written
    assert c0.numel() == 0 and v0.shape == (1, 0)
    c1, v1 = B.fill_rows(rowptr, 7, 8, T)                    # one row
    assert torch.equal(c1, col[rp[7]:rp[8]]) and torch.equal(v1, val[:, rp[7]:rp[8]])
    c2, v2 = B.fill_rows(rowptr, B.dim - 1, B.dim, T)        # the last row
    assert torch.equal(c2, col[rp[-2]:]) and torch.equal(v2, val[:, rp[-2]:])
    B.check()
    with pytest.raises(ValueError):
        B.fill_rows(rowptr, 5, 4, T)
    import ctypes as C                                       # the C entry's own range check
    assert cih.lib.cih_ham_fill_rows(B._h, C.c_void_p(rowptr.data_ptr()), 5, 4, 1, 20.0, C.c_void_p(T.data_ptr()),
                                     None, C.c_void_p(col.data_ptr()), C.c_void_p(val.data_ptr()), None) == -1
