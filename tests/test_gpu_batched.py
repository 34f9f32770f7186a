"""GPU: K interaction sets sharing one structure (4+4 Nmax=4, 2M=0, K=64).

- the set-major fill, the fill from interleaved tables and the batched fill
  (element-major values) agree bit for bit; against K independent single-set
  fills the structure is bit-identical and the values agree within 1e-6
  (multi-term values are summed in term order per set, the single-set fill
  sums them as a warp tree);
- sampled rows of two sets agree with the oracle;
- every launch shape the autotuner tries gives the same bits;
- count + scan + fill captured in one CUDA graph and replayed agree with the
  eager calls;
- the K Krylov sequences advancing together give each set's eigenvalues as
  a single-set Lanczos does, and one set against the oracle's Lanczos.
"""
import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SP = (4, 4, 4, 0)
K = 64
SEEDS = list(range(1000, 1000 + K))


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.fixture(scope="module")
def built(cih):
    B = cih.Basis(*SP)
    T = torch.from_numpy(synth.tbme_tables(B.tbme_len, SEEDS)).cuda()
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, T)
    B.check()
    yield B, T, rowptr, nnz, col, val
    del col, val
    torch.cuda.empty_cache()


def test_interleaved_equals_set_major(cih, built):
    B, T, rowptr, nnz, col, val = built
    til = cih.tbme_interleave(T)
    np.testing.assert_array_equal(til.view(B.tbme_len, K)[:, 5].cpu().numpy(), T[5].cpu().numpy())
    col2, val2 = B.fill_interleaved(rowptr, nnz, til, K)
    B.check()
    assert torch.equal(col2, col)
    assert torch.equal(val2, val)
    del col2, val2, til


def test_batched_element_major(cih, built):
    B, T, rowptr, nnz, col, val = built
    til = cih.tbme_interleave(T)
    c3, vem = B.fill_batched(rowptr, nnz, til, K)
    B.check()
    assert vem.shape == (nnz, K)
    assert torch.equal(c3, col)
    assert torch.equal(vem.t(), val)
    del c3, vem, til


@pytest.mark.parametrize("k", [0, 17, 63])
def test_batched_equals_single(cih, built, k):
    B, T, rowptr, nnz, col, val = built
    c1, v1 = B.fill(rowptr, nnz, T[k].contiguous())
    assert torch.equal(c1, col)
    a, b = v1[0].double(), val[k].double()
    assert torch.all((a - b).abs() <= 1e-6 * (b.abs() + 1.0))
    assert (a == b).double().mean() > 0.999


def test_batched_sampled_rows_against_oracle(cih, built):
    B, T, rowptr, nnz, col, val = built
    S = oracle.Space(*SP)
    rp = rowptr.cpu().numpy()
    c = col.cpu().numpy()
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([[0, B.dim - 1], rng.integers(0, B.dim, 120)])).astype(np.int64)
    for k in (1, 62):
        t = T[k].cpu().numpy()
        cnt, off, col_o, val_o = S.rows(rows, t)
        v = val[k].cpu().numpy()
        np.testing.assert_array_equal(np.diff(rp)[rows], cnt)
        np.testing.assert_array_equal(np.concatenate([c[rp[r]:rp[r + 1]] for r in rows]), col_o)
        got = np.concatenate([v[rp[r]:rp[r + 1]] for r in rows]).astype(np.float64)
        assert np.all(np.abs(got - val_o) <= 1e-5 * (np.abs(val_o) + 1.0))


def test_launch_shapes_and_autotuner(cih, built):
    B, T, rowptr, nnz, col, val = built
    T8 = T[:8].contiguous()
    ref_c, ref_v = B.fill(rowptr, nnz, T8)
    for warps, ctas in [(8, 0), (8, 1), (16, 1), (16, 2)]:
        B.set_launch(warps, ctas)
        c2, v2 = B.fill(rowptr, nnz, T8)
        assert torch.equal(c2, ref_c) and torch.equal(v2, ref_v), (warps, ctas)
    c3, v3, (w, ct, ms) = B.autotune_fill(rowptr, nnz, T8)
    assert w in (8, 16) and 0 <= ct <= 3 and ms > 0
    assert torch.equal(c3, ref_c) and torch.equal(v3, ref_v)
    til = cih.tbme_interleave(T8)
    c4, v4, _ = B.autotune_fill(rowptr, nnz, til, K=8, interleaved=True)
    assert torch.equal(c4, ref_c) and torch.equal(v4, ref_v)
    c5, v5, _ = B.autotune_fill(rowptr, nnz, til, K=8, batched=True)
    assert torch.equal(c5, ref_c) and torch.equal(v5.t(), ref_v)
    B.set_launch(16, 0)
    with pytest.raises(cih.CihError):
        B.set_launch(12, 0)


def test_graph_capture_replay(cih, built):
    """count + scan + fill of the K sets captured once, replayed twice."""
    B, T, rowptr, nnz, col, val = built
    s = torch.cuda.Stream()
    rp = torch.empty_like(rowptr)
    c = torch.empty_like(col)
    v = torch.empty_like(val)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):                               # warm-up outside the capture
        B.count_into(rp, stream=s)
        B.fill(rp, nnz, T, stream=s, col=c, val=v)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    rp.zero_()
    c.zero_()
    v.zero_()
    torch.cuda.synchronize()
    before = cih.kernel_launches()
    with torch.cuda.graph(g, stream=s):
        B.count_into(rp, stream=s)
        B.fill(rp, nnz, T, stream=s, col=c, val=v)
    captured = cih.kernel_launches() - before
    assert captured >= 3                                     # count, scan (>= 1), fill
    for _ in range(2):
        v.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(rp, rowptr)
        assert torch.equal(c[:nnz], col) and torch.equal(v[:, :nnz], val)
    B.check()
    del g, v
    # the batched fill (interleaved tables, element-major values) in a graph
    til = cih.tbme_interleave(T)
    vem = torch.empty((nnz, K), dtype=torch.float32, device="cuda")
    with torch.cuda.stream(s):
        B.fill_batched(rp, nnz, til, K, stream=s, col=c, val=vem)
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2, stream=s):
        B.count_into(rp, stream=s)
        B.fill_batched(rp, nnz, til, K, stream=s, col=c, val=vem)
    vem.zero_()
    g2.replay()
    torch.cuda.synchronize()
    assert torch.equal(vem.t(), val)
    B.check()
    del g2, vem, til


def test_batched_lanczos(cih, built):
    B, T, rowptr, nnz, col, val = built
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=400, tol=1e-9)
    assert conv
    assert ev.shape == (K, 5) and np.all(np.diff(ev, axis=1) >= -1e-9)
    # the same from the batched fill's element-major values, read in place
    til = cih.tbme_interleave(T)
    c3, vem = B.fill_batched(rowptr, nnz, til, K)
    ev_em, psi_em, conv_em = B.lanczos(rowptr, c3, vem, nev=5, max_iter=400, tol=1e-9, element_major=True)
    assert conv_em
    np.testing.assert_array_equal(ev_em, ev)
    assert torch.equal(psi_em, psi)
    del c3, vem, til, psi_em
    # each set as a single-set run (same start vector; sums in another order)
    for k in (0, 31, 63):
        ev1, psi1, conv1 = B.lanczos(rowptr, col, val[k:k + 1], nev=5, max_iter=400, tol=1e-9)
        assert conv1
        np.testing.assert_allclose(ev[k], ev1[0], rtol=1e-9, atol=1e-9)
        ov = abs(float(torch.dot(psi[k], psi1[0])))
        assert ov == pytest.approx(1.0, abs=1e-6)
    # one set against the oracle's Lanczos on the same stored matrix
    k = 40
    ev_o, _, _, conv_o = oracle.lanczos(rowptr.cpu().numpy(), col.cpu().numpy(), val[k].cpu().numpy(),
                                        nev=5, max_iter=400, tol=1e-12)
    assert conv_o
    np.testing.assert_allclose(ev[k], ev_o, rtol=1e-5)
    # the Ritz vectors are normalised eigenvectors: residual of set 7 by one more product
    p = psi[7].cpu().numpy()
    assert abs(np.linalg.norm(p) - 1.0) < 1e-10
    del psi
    torch.cuda.empty_cache()


def test_batched_four_word_strings_against_oracle(cih):
    """The 64-set batched kernel on a space whose sub-determinants take four
    64-bit words (3+3 Nmax=6: 60 M stored nonzeros, 15.4 GB of values):
    sampled rows of the first and last set against the oracle."""
    sp = (3, 3, 6, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    T = synth.tbme_tables(B.tbme_len, SEEDS)
    til = cih.tbme_interleave(torch.from_numpy(T).cuda())
    rowptr, nnz = B.count()
    col, vem = B.fill_batched(rowptr, nnz, til, K)
    B.check()
    rp = rowptr.cpu().numpy()
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([rng.integers(0, B.dim, 40), [0, B.dim - 1]])).astype(np.int64)
    c = col.cpu().numpy()
    sel = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    v_sel = vem[torch.from_numpy(sel).cuda()].cpu().numpy()                 # (elements, K)
    for k in (0, K - 1):
        cnt, off, col_o, val_o = S.rows(rows, T[k])
        np.testing.assert_array_equal(np.diff(rp)[rows], cnt)
        np.testing.assert_array_equal(c[sel], col_o)
        v = v_sel[:, k].astype(np.float64)
        bad = np.abs(v - val_o) > 1e-5 * (np.abs(val_o) + 1.0)
        assert not bad.any(), (k, int(bad.sum()))
    del col, vem, til
    torch.cuda.empty_cache()
