"""GPU: the fill with a one-body table (cih_ham_fill_onebody) against the
oracle with the same table (Sec. 2: the one-body operator read from file).

The one-body table is synthetic: standard-normal entries in table order, with
hbar_omega (N_a + 3/2) added to each diagonal t_aa, so that the off-diagonal
couplings (Delta N = 0 and 2) perturb an oscillator spectrum.  Structure is
compared bit-exact, values within 1e-5 (|oracle| + 1), eigenvalues within
1e-5 relative."""
import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VTOL = 1e-5


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


def onebody(S, seed):
    t1 = synth.onebody_table(S.onebody_len, seed)
    o = np.concatenate([S.orbitals(0), S.orbitals(1)])
    for a in range(len(o)):
        t1[S.onebody_index(a, a)] += 20.0 * (o[a, 0] + 1.5)
    return t1


def assert_values(v_gpu, v_or):
    v_gpu = np.asarray(v_gpu, dtype=np.float64)
    v_or = np.asarray(v_or, dtype=np.float64)
    bad = np.abs(v_gpu - v_or) > VTOL * (np.abs(v_or) + 1.0)
    assert not bad.any(), f"{bad.sum()} values out of tolerance, first at {np.nonzero(bad)[0][:5]}"


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (2, 2, 2, 0), (2, 1, 3, 1), (1, 0, 3, 1), (2, 0, 2, 0),
                                (3, 3, 4, 0), (3, 2, 2, 3)])
def test_whole_matrix(cih, sp):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t1 = onebody(S, 2)
    T = synth.tbme_tables(B.tbme_len, [3, 4])
    rowptr, nnz = B.count()
    col, val = B.fill_onebody(rowptr, nnz, torch.from_numpy(T).cuda(), t1)
    B.check()
    S.set_onebody(t1)
    for k in range(2):
        rp_o, col_o, val_o = S.half_csr(T[k])
        np.testing.assert_array_equal(rowptr.cpu().numpy(), rp_o)
        np.testing.assert_array_equal(col.cpu().numpy(), col_o)
        assert_values(val[k].cpu().numpy(), val_o)


@pytest.mark.parametrize("sp,nsample", [((3, 3, 6, 0), 150), ((4, 4, 6, 0), 100)])
def test_sampled_rows_full_size(cih, sp, nsample):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t1 = onebody(S, 5)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, nnz = B.count()
    col, val = B.fill_onebody(rowptr, nnz, torch.from_numpy(t).cuda(), t1)
    B.check()
    rp = rowptr.cpu().numpy()
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.integers(0, B.dim, nsample), [0, B.dim - 1]])).astype(np.int64)
    S.set_onebody(t1)
    cnt, off, col_o, val_o = S.rows(rows, t)
    np.testing.assert_array_equal(np.diff(rp)[rows], cnt)
    c, v = col.cpu().numpy(), val[0].cpu().numpy()
    np.testing.assert_array_equal(np.concatenate([c[rp[r]:rp[r + 1]] for r in rows]), col_o)
    assert_values(np.concatenate([v[rp[r]:rp[r + 1]] for r in rows]), val_o)
    del col, val
    torch.cuda.empty_cache()


def test_lanczos_with_onebody_table_against_dense(cih):
    sp = (3, 3, 2, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t1 = onebody(S, 7)
    t = synth.tbme_table(B.tbme_len, 1)
    rowptr, nnz = B.count()
    col, val = B.fill_onebody(rowptr, nnz, torch.from_numpy(t).cuda(), t1)
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=300, tol=1e-10)
    assert conv
    S.set_onebody(t1)
    w = np.linalg.eigvalsh(S.dense_sc(t))
    np.testing.assert_allclose(ev[0], w[:5], rtol=1e-5)
