"""GPU parity of the half-stored matrix-vector product y = H x (cih_ham_spmv,
the product Lanczos applies, Sec. 2) against the oracle's product.

The library reads each stored nonzero once, with no FP64 operation per
nonzero: products of a value and an FP32-pair copy of x (relative error about
2^-47), the row part a double-float sum, the mirrored part in 64-bit fixed
point (units 2^-s, 2^s <= 2^60 / (F ||x||), F the Frobenius norm of the
strictly-upper values), each mirrored product rounded by at most one unit.  A
column of c terms is then off by at most c 2^-60 F ||x|| plus 2^-46 of its
terms' magnitudes: the tolerance below, 1e-11 max |y|, holds that with room
at these sizes.
"""
import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


def assert_close(y, want):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - want).max()
    assert err <= 1e-11 * np.abs(want).max() + 1e-300, err


def built(cih, sp, seeds):
    B = cih.Basis(*sp)
    T = synth.tbme_tables(B.tbme_len, seeds)
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, torch.from_numpy(T).cuda())
    B.check()
    return B, rowptr, nnz, col, val


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (2, 1, 3, 1), (3, 3, 4, 0)])
def test_one_set_against_oracle(cih, sp):
    B, rowptr, nnz, col, val = built(cih, sp, [5])
    x = np.random.default_rng(2).standard_normal(B.dim)            # not normalised
    y = B.spmv(rowptr, col, val, torch.from_numpy(x).cuda())
    B.check()
    want = oracle.half_spmv(rowptr.cpu().numpy(), col.cpu().numpy(), val[0].cpu().numpy(), x)
    assert_close(y.cpu().numpy(), want)
    y2 = B.spmv(rowptr, col, val, torch.from_numpy(x).cuda())       # deterministic
    assert torch.equal(y, y2)


def test_sets_and_layouts(cih):
    """K = 3 (set-major), the same from element-major values, and each set
    against the oracle."""
    sp = (3, 3, 4, 0)
    B, rowptr, nnz, col, val = built(cih, sp, [1, 2, 3])
    K = 3
    x = np.random.default_rng(4).standard_normal((B.dim, K))
    xd = torch.from_numpy(x).cuda()
    y = B.spmv(rowptr, col, val, xd)
    y_em = B.spmv(rowptr, col, val.t().contiguous(), xd, element_major=True)
    assert torch.equal(y, y_em)
    rp, c = rowptr.cpu().numpy(), col.cpu().numpy()
    for k in range(K):
        assert_close(y[:, k].cpu().numpy(), oracle.half_spmv(rp, c, val[k].cpu().numpy(), x[:, k]))


def test_batched_values_in_place(cih):
    """K = 64 element-major values from the batched fill, read in place."""
    sp = (3, 3, 2, 0)
    B = cih.Basis(*sp)
    K = 64
    T = synth.tbme_tables(B.tbme_len, list(range(K)))
    rowptr, nnz = B.count()
    col, vem = B.fill_batched(rowptr, nnz, cih.tbme_interleave(torch.from_numpy(T).cuda()), K)
    B.check()
    x = np.random.default_rng(6).standard_normal((B.dim, K))
    y = B.spmv(rowptr, col, vem, torch.from_numpy(x).cuda(), element_major=True)
    rp, c, v = rowptr.cpu().numpy(), col.cpu().numpy(), vem.cpu().numpy()
    for k in (0, 17, 63):
        assert_close(y[:, k].cpu().numpy(), oracle.half_spmv(rp, c, v[:, k], x[:, k]))


def test_degenerate_inputs(cih):
    """A zero two-body table (only the diagonal is nonzero: F = 0), a vector
    of entries near 1e150 (the scale goes far below 1), and an empty basis."""
    sp = (3, 3, 2, 0)
    B = cih.Basis(*sp)
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, torch.zeros((1, B.tbme_len), device="cuda"))
    x = np.random.default_rng(7).standard_normal(B.dim)
    y = B.spmv(rowptr, col, val, torch.from_numpy(x).cuda()).cpu().numpy()
    d = val[0].cpu().numpy()[rowptr.cpu().numpy()[:-1]].astype(np.float64)
    np.testing.assert_allclose(y, d * x, rtol=1e-13, atol=0)
    B2, rowptr2, nnz2, col2, val2 = built(cih, sp, [9])
    xb = 1e150 * np.random.default_rng(8).standard_normal(B2.dim)
    yb = B2.spmv(rowptr2, col2, val2, torch.from_numpy(xb).cuda())
    assert_close(yb.cpu().numpy(), oracle.half_spmv(rowptr2.cpu().numpy(), col2.cpu().numpy(),
                                                     val2[0].cpu().numpy(), xb))
    E = cih.Basis(2, 2, 2, 1)                                      # no state with 2M = 1
    assert E.dim == 0
    rpe, _ = E.count()
    ye = E.spmv(rpe, torch.zeros(1, dtype=torch.int32, device="cuda"), torch.zeros((1, 1), device="cuda"),
                torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert ye.numel() == 0


@pytest.mark.parametrize("sp", [(3, 3, 6, 0), (4, 4, 6, 0)])
def test_full_size_against_oracle(cih, sp):
    """3+3 Nmax=6 (60 M stored nonzeros) and 4+4 Nmax=6 (925 M): the whole
    product, the launch configuration the benchmark times, against the
    oracle's product on the copied matrix, with a unit vector as Lanczos
    applies it."""
    B = cih.Basis(*sp)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    B.check()
    x = np.random.default_rng(10).standard_normal(B.dim)
    x /= np.linalg.norm(x)
    y = B.spmv(rowptr, col, val, torch.from_numpy(x).cuda()).cpu().numpy()
    B.check()
    rp, c, v = rowptr.cpu().numpy(), col.cpu().numpy(), val[0].cpu().numpy()
    del col, val
    torch.cuda.empty_cache()
    assert_close(y, oracle.half_spmv(rp, c, v, x))
