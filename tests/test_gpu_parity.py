"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Structure (row pointers, columns) must be bit-exact; values agree within
|gpu - oracle| <= 1e-5 (|oracle| + 1) (the documented bound: FP32 storage of
FP64 sums of FP32 table entries; in practice the values are bit-identical);
eigenvalues within 1e-5 relative; gradients within 1e-9 absolute (the
fixed-point accumulator resolves 2^-56).

Small spaces are compared whole.  At the benchmark sizes the oracle computes
sampled rows one by one (first, last, random, ragged ends of proton blocks),
and whole-matrix properties (row counts sum to nnz, columns ascending and
>= the row, diagonal first) are checked on every row.
"""
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


def assert_values(v_gpu, v_or):
    v_gpu = np.asarray(v_gpu, dtype=np.float64)
    v_or = np.asarray(v_or, dtype=np.float64)
    bad = np.abs(v_gpu - v_or) > VTOL * (np.abs(v_or) + 1.0)
    assert not bad.any(), f"{bad.sum()} values out of tolerance, first at {np.nonzero(bad)[0][:5]}"


SMALL = [(3, 3, 2, 0), (2, 2, 2, 0), (2, 1, 3, 1), (1, 1, 2, 0), (2, 0, 2, 0), (0, 2, 2, 0),
         (3, 3, 2, 8), (1, 0, 3, 1), (2, 2, 0, 0), (3, 0, 2, 1), (2, 2, 3, 8), (3, 3, 3, 1)]


@pytest.mark.parametrize("sp", SMALL)
def test_whole_matrix_small(cih, sp):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    assert B.dim == S.dim and B.tbme_len == S.tbme_len
    t = synth.tbme_table(B.tbme_len, 11)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    B.check()
    rp_o, col_o, val_o = S.half_csr(t)
    assert nnz == rp_o[-1]
    np.testing.assert_array_equal(rowptr.cpu().numpy(), rp_o)
    np.testing.assert_array_equal(col.cpu().numpy(), col_o)
    assert_values(val[0].cpu().numpy(), val_o)


def test_whole_matrix_mid(cih):
    """3+3 Nmax=4: several thousand rows, every proton-block shape, ragged tails."""
    sp = (3, 3, 4, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t = synth.tbme_table(B.tbme_len, 5)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    B.check()
    rp_o, col_o, val_o = S.half_csr(t)
    np.testing.assert_array_equal(rowptr.cpu().numpy(), rp_o)
    np.testing.assert_array_equal(col.cpu().numpy(), col_o)
    assert_values(val[0].cpu().numpy(), val_o)


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (2, 1, 3, 1), (3, 3, 4, 0), (4, 4, 4, 0)])
def test_count_walk_against_oracle(cih, sp):
    """The count pass's walk form -- the one a basis without count lists
    (bucket directory above 4096 entries, or above 63 levels) runs -- selected
    with cih_set_count_mode: row counts equal to the oracle's, row pointers
    equal to the count-list form's."""
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    rp_lists, nnz_lists = B.count()
    B.set_count_mode(True)
    rp_walk, nnz_walk = B.count()
    B.check()
    B.set_count_mode(False)
    np.testing.assert_array_equal(np.diff(rp_walk.cpu().numpy()), S.count_rows())
    assert nnz_walk == nnz_lists and torch.equal(rp_walk, rp_lists)


def test_empty_basis(cih):
    B = cih.Basis(2, 2, 2, 1)
    assert B.dim == 0
    rowptr, nnz = B.count()
    assert nnz == 0 and rowptr.cpu().tolist() == [0]


def test_multiple_sets_and_one_body_override(cih):
    sp = (2, 2, 2, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    T = synth.tbme_tables(B.tbme_len, range(3))
    esp = synth.single_particle_energies(sum(B.n_orb), 4)
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, torch.from_numpy(T).cuda(), e_sp=torch.from_numpy(esp))
    B.check()
    for k in range(3):
        rp_o, col_o, val_o = S.half_csr(T[k], esp)
        np.testing.assert_array_equal(col.cpu().numpy(), col_o)
        assert_values(val[k].cpu().numpy(), val_o)


def test_closed_form_tables(cih):
    """Zero table: diagonal HO sums; unit-diagonal table: + A(A-1)/2, no off-diagonal."""
    sp = (3, 3, 2, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    z = np.zeros(B.tbme_len, np.float32)
    u = z.copy()
    for c in range(3):
        pa, pb, _ = S.channel_pairs(c)
        for a, b in zip(pa, pb):
            u[S.tbme_index(int(a), int(b), int(a), int(b))[0]] = 1.0
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, torch.from_numpy(np.stack([z, u])).cuda())
    rp = rowptr.cpu().numpy()
    c = col.cpu().numpy()
    v = val.cpu().numpy()
    diag = rp[:-1]
    assert np.all(c[diag] == np.arange(B.dim))
    off = np.ones(nnz, bool)
    off[diag] = False
    assert np.all(v[0][off] == 0) and np.all(v[1][off] == 0)
    assert sorted(set(v[0][diag].tolist())) == [220.0, 260.0]
    np.testing.assert_array_equal(v[1][diag], v[0][diag] + 15.0)


def check_structure(rp, col):
    dim = len(rp) - 1
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1)
    rows = np.repeat(np.arange(dim), np.diff(rp))
    assert np.all(col >= rows)
    assert np.all(col[rp[:-1]] == np.arange(dim))            # diagonal first
    inner = np.ones(len(col), bool)
    inner[rp[:-1]] = False                                   # first entry of each row
    d = np.diff(col.astype(np.int64))
    assert np.all(d[inner[1:]] > 0)                           # ascending inside rows


def sample_rows(B, n_random, seed):
    t = B.tables()
    rb = t["rowbase"]
    rng = np.random.default_rng(seed)
    rows = set(rng.integers(0, B.dim, size=n_random).tolist())
    rows |= {0, 1, B.dim - 1, B.dim - 2}
    ps = rng.integers(0, len(rb) - 1, size=16)
    for p in ps:                                             # ends of proton blocks
        rows |= {int(rb[p]), int(rb[p + 1] - 1)}
    return np.array(sorted(r for r in rows if 0 <= r < B.dim), dtype=np.int64)


@pytest.mark.parametrize("sp,nsample", [((4, 4, 4, 0), 300), ((5, 6, 4, 1), 200), ((3, 3, 6, 0), 200),
                                        ((4, 4, 6, 0), 120)])
def test_sampled_rows_full_size(cih, sp, nsample):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    assert B.dim == S.dim
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    B.check()
    rp = rowptr.cpu().numpy()
    c = col.cpu().numpy()
    check_structure(rp, c)
    v = val[0].cpu().numpy()
    rows = sample_rows(B, nsample, 7)
    cnt, off, col_o, val_o = S.rows(rows, t)
    np.testing.assert_array_equal(np.diff(rp)[rows], cnt)
    got_c = np.concatenate([c[rp[r]:rp[r + 1]] for r in rows])
    got_v = np.concatenate([v[rp[r]:rp[r + 1]] for r in rows])
    np.testing.assert_array_equal(got_c, col_o)
    assert_values(got_v, val_o)
    del col, val
    torch.cuda.empty_cache()


def test_lanczos_small_against_dense(cih):
    sp = (3, 3, 2, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=300, tol=1e-10)
    assert conv
    rp_o, col_o, val_o = S.half_csr(t)
    H = np.zeros((S.dim, S.dim))
    for i in range(S.dim):
        H[i, col_o[rp_o[i]:rp_o[i + 1]]] = val_o[rp_o[i]:rp_o[i + 1]]
    H = H + np.triu(H, 1).T
    w = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(ev[0], w[:5], rtol=1e-5)
    p = psi[0].cpu().numpy()
    assert abs(np.linalg.norm(p) - 1) < 1e-10
    assert np.linalg.norm(H @ p - ev[0][0] * p) < 1e-6 * np.abs(w).max()


def test_lanczos_degenerate_zero_table(cih):
    B = cih.Basis(3, 3, 2, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.zeros((1, B.tbme_len), device="cuda"))
    ev, _, conv = B.lanczos(rowptr, col, val, nev=2, max_iter=50, tol=1e-10)
    assert conv
    np.testing.assert_allclose(ev[0], [220.0, 260.0], rtol=1e-12)


def test_lanczos_mid_against_oracle(cih):
    sp = (4, 4, 4, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=400, tol=1e-9)
    assert conv
    ev_o, _, _, conv_o = oracle.lanczos(rowptr.cpu().numpy(), col.cpu().numpy(), val[0].cpu().numpy(),
                                        nev=5, max_iter=400, tol=1e-12)
    assert conv_o
    np.testing.assert_allclose(ev[0], ev_o, rtol=1e-5)


@pytest.mark.parametrize("sp", [(2, 2, 2, 0), (3, 3, 2, 0), (2, 1, 3, 1)])
def test_gradient_against_oracle(cih, sp):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t = synth.tbme_table(B.tbme_len, 9)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    rp_o, col_o, val_o = S.half_csr(t)
    H = S.dense_sc(t)
    w, V = np.linalg.eigh(H)
    psi = V[:, 0]
    g = B.tbme_grad(rowptr, torch.from_numpy(psi).cuda())[0].cpu().numpy()
    g_o = S.grad_elementwise(rp_o, col_o, psi)
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-9)
    # and the brute-force two-body density
    np.testing.assert_allclose(g, S.density_brute(psi), rtol=0, atol=1e-9)


def test_gradient_full_path_mid(cih):
    """4+4 Nmax=4: GPU Lanczos vector -> GPU adjoint vs oracle adjoint on the same vector."""
    sp = (4, 4, 4, 0)
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=1, max_iter=400, tol=1e-9)
    assert conv
    g = B.tbme_grad(rowptr, psi)[0].cpu().numpy()
    g_o = S.grad_elementwise(rowptr.cpu().numpy(), col.cpu().numpy(), psi[0].cpu().numpy())
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-9)
    # Euler identity: E0 = <one-body> + sum_t g_t t  (H linear in the table)
    rp0, col0, val0, _ = cih.build_hamiltonian(B, torch.zeros((1, B.tbme_len), device="cuda"))
    p = psi[0].cpu().numpy()
    diag = val0[0].cpu().numpy()[rp0.cpu().numpy()[:-1]]
    e1 = float(np.sum(diag * p * p))
    assert e1 + float(g @ t.astype(np.float64)) == pytest.approx(ev[0][0], rel=1e-6)


def _torch_lanczos(matvec, dim, nev, iters, seed):
    """Plain FP64 Lanczos in torch with full reorthogonalisation (classical
    Gram-Schmidt twice) from a seeded normal start: the nev lowest Ritz
    values and vectors of the last step, and the residual bounds."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.randn(dim, dtype=torch.float64, device="cuda", generator=g)
    V = torch.empty((iters + 1, dim), dtype=torch.float64, device="cuda")
    V[0] = v / torch.linalg.vector_norm(v)
    al, be = [], []
    m = 0
    for j in range(iters):
        w = matvec(V[j])
        for _ in range(2):
            h = V[: j + 1] @ w
            w -= V[: j + 1].T @ h
            if _ == 0:
                al.append(float(h[j]))
            else:
                al[-1] += float(h[j])
        b = float(torch.linalg.vector_norm(w))
        m = j + 1
        if b < 1e-12:
            break
        be.append(b)
        V[j + 1] = w / b
        if m >= nev and m % 20 == 0:                 # stop once the nev residual bounds are small
            T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
            th, Z = np.linalg.eigh(T)
            if np.all(b * np.abs(Z[-1, :nev]) <= 1e-8 * np.abs(th[:nev])):
                break
    T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
    th, Z = np.linalg.eigh(T)
    Y = torch.from_numpy(Z[:, :nev].copy()).cuda().T @ V[:m]
    return th[:nev], Y


def test_lanczos_residual_full_size(cih):
    """4+4 Nmax=6 (925 M stored nonzeros), too large for the oracle's Lanczos.
    The library's five lowest eigenvalues against an independent FP64 Lanczos
    in torch whose products are built from the stored half (row part +
    mirrored part - diagonal); the true residual |H y - theta y| of each of
    that run's five lowest Ritz pairs, and of the library's lowest Ritz vector."""
    sp = (4, 4, 6, 0)
    B = cih.Basis(*sp)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=600, tol=1e-9)
    assert conv
    v = val[0].double()
    del val
    rows = torch.repeat_interleave(torch.arange(B.dim, device="cuda"), rowptr[1:] - rowptr[:-1])
    c = col.long()
    del col
    diag = rowptr[:-1]
    vd = v[diag]

    def matvec(x):
        y = torch.zeros(B.dim, dtype=torch.float64, device="cuda")
        y.index_add_(0, rows, v * x[c])                              # upper half
        y.index_add_(0, c, v * x[rows])                              # mirrored half
        return y - vd * x                                            # the diagonal counted once

    x = psi[0]
    assert abs(float(torch.linalg.vector_norm(x)) - 1.0) < 1e-10
    res0 = float(torch.linalg.vector_norm(matvec(x) - ev[0][0] * x))
    assert res0 <= 1e-6 * abs(ev[0][0]), res0
    th, Y = _torch_lanczos(matvec, B.dim, 5, 400, 11)
    for k in range(5):
        y = Y[k] / torch.linalg.vector_norm(Y[k])
        res = float(torch.linalg.vector_norm(matvec(y) - th[k] * y))
        assert res <= 1e-5 * abs(th[k]), (k, res)
    np.testing.assert_allclose(ev[0], th, rtol=1e-5)
    del rows, c, v, Y
    torch.cuda.empty_cache()


def test_lanczos_5p6n_against_oracle(cih):
    """5+6 Nmax=4, 2M=1 (the uneven batch's third instance, seed 102; 207 M
    stored nonzeros): the library's five lowest eigenvalues against the
    oracle's Lanczos run on the GPU-built matrix."""
    sp = (5, 6, 4, 1)
    B = cih.Basis(*sp)
    t = synth.tbme_table(B.tbme_len, 102)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    B.check()
    ev, _, conv = B.lanczos(rowptr, col, val, nev=5, max_iter=500, tol=1e-9)
    assert conv
    ev_o, _, _, conv_o = oracle.lanczos(rowptr.cpu().numpy(), col.cpu().numpy(), val[0].cpu().numpy(),
                                        nev=5, max_iter=500, tol=1e-10)
    assert conv_o
    np.testing.assert_allclose(ev[0], ev_o, rtol=1e-5)
    del col, val
    torch.cuda.empty_cache()
