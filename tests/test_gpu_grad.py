"""GPU: d(lowest eigenvalue)/d(two-body table) at 4+4 Nmax=4, 2M=0, one table.

The adjoint (Hellmann-Feynman: g_t = sum over stored elements using t of
w * phase * psi_i psi_j) through torch.autograd, against

- central finite differences of the lowest eigenvalue on 32 random table
  entries, the 64 perturbed tables built and solved as one batch of K = 64
  sets sharing the structure;
- central FP64 differences on 8 entries: H is linear in each entry, so
  E0(H +- h dH/dt_k) is taken with an FP64 Lanczos in torch on the stored
  matrix plus or minus h times the exact (0, +-1) fill of that entry, within
  1e-6 (test_fp64_central_differences);
- the oracle's adjoint walk (its two-body density of psi) on the same vector;
- the Euler identity E0 = <one-body> + sum_t g_t t (H is linear in the table).

Finite-difference error budget for step h = 2^-6 (t +- h exact in FP32
unless |t| < h; the quotient uses the step actually taken): truncation
h^2/6 |E'''|, |E'''| <~ 8 |dH|^3 / gap^2 with |dH| <= 2, gives < 1e-4 for
gaps above ~2 MeV; the FP32 rounding of
stored values (|delta| <= 2^-24 |v|, |v| <~ 300 MeV on the diagonal, weighted
by psi_i^2 summing to <= 1) adds at most 2 * 1.8e-5 / (2h) = 1.1e-3.  Hence
|FD - g| <= 2e-3.
"""
import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SP = (4, 4, 4, 0)
H_STEP = 2.0 ** -6
FD_ATOL = 2e-3


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


def test_autograd_fd_density_euler(cih):
    B = cih.Basis(*SP)
    t_np = synth.tbme_table(B.tbme_len, 0)
    t = torch.from_numpy(t_np).cuda().requires_grad_(True)
    e0 = cih.lowest_eigenvalue(B, t, max_iter=500, tol=1e-11)
    e0.backward()
    g32 = t.grad.detach().cpu().numpy()

    # the FP64 adjoint behind the autograd function
    rowptr, col, val, nnz = cih.build_hamiltonian(B, t.detach().unsqueeze(0))
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=1, max_iter=500, tol=1e-11)
    assert conv
    assert float(e0.detach()) == ev[0][0]
    g = B.tbme_grad(rowptr, psi)[0].cpu().numpy()
    np.testing.assert_array_equal(g32, g.astype(np.float32))
    assert np.all(np.abs(g) <= 2.0 + 1e-12)

    # oracle: its adjoint walk on the same vector
    S = oracle.Space(*SP)
    g_o = S.grad_elementwise(rowptr.cpu().numpy(), col.cpu().numpy(), psi[0].cpu().numpy())
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-9)

    # Euler identity
    rp0, col0, val0, _ = cih.build_hamiltonian(B, torch.zeros((1, B.tbme_len), device="cuda"))
    p = psi[0].cpu().numpy()
    diag = val0[0].cpu().numpy()[rp0.cpu().numpy()[:-1]]
    e1 = float(np.sum(diag * p * p))
    assert e1 + float(g @ t_np.astype(np.float64)) == pytest.approx(ev[0][0], rel=1e-6)
    del col, val, col0, val0

    # central differences on 32 random entries, as one K = 64 batch
    rng = np.random.default_rng(11)
    idx = rng.choice(B.tbme_len, size=32, replace=False)
    T = np.repeat(t_np[None, :], 64, axis=0)
    for q, k in enumerate(idx):
        T[2 * q, k] += np.float32(H_STEP)
        T[2 * q + 1, k] -= np.float32(H_STEP)
    step = T[0::2][np.arange(32), idx].astype(np.float64) - T[1::2][np.arange(32), idx].astype(np.float64)
    assert np.all(np.abs(step - 2 * H_STEP) <= 1e-6)         # exact unless |t| < h (then rounded)
    Tt = torch.from_numpy(T).cuda()
    rowptr2, nnz2 = B.count()
    col2, val2 = B.fill(rowptr2, nnz2, Tt)
    evk, _, convk = B.lanczos(rowptr2, col2, val2, nev=1, max_iter=500, tol=1e-11, want_vectors=False)
    assert convk
    fd = (evk[0::2, 0] - evk[1::2, 0]) / step
    err = np.abs(fd - g[idx])
    assert err.max() <= FD_ATOL, (err.max(), idx[np.argmax(err)])


def test_adjoint_flags_an_unnormalised_vector(cih):
    """A vector of squared norm 4 (every entry far below the per-entry bound
    of 4) would let the fixed-point sums outgrow their range: the adjoint
    sets the device status, which cih_check reports and clears."""
    B = cih.Basis(2, 2, 2, 0)
    t = torch.from_numpy(synth.tbme_table(B.tbme_len, 3)).cuda()
    rowptr, col, val, nnz = cih.build_hamiltonian(B, t)
    B.check()
    psi = torch.full((B.dim,), 2.0 / np.sqrt(B.dim), dtype=torch.float64, device="cuda")
    B.tbme_grad(rowptr, psi)
    with pytest.raises(cih.CihError, match="status bits 32"):
        B.check()
    B.tbme_grad(rowptr, psi / 2.0)                           # normalised: no flag
    B.check()


def _fp64_lowest(rows, c, vals, vd, dim, seed, tol=1e-9, iters=600):
    """Lowest eigenvalue of the half-stored FP64 matrix (vals) by a plain FP64
    Lanczos in torch with full reorthogonalisation (classical Gram-Schmidt
    twice), from a seeded normal start, stopped when the residual bound of
    the lowest Ritz pair is below tol |theta|."""
    def mv(x):
        y = torch.zeros(dim, dtype=torch.float64, device="cuda")
        y.index_add_(0, rows, vals * x[c])                         # upper half
        y.index_add_(0, c, vals * x[rows])                         # mirrored half
        return y - vd * x                                          # the diagonal counted once
    g = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.randn(dim, dtype=torch.float64, device="cuda", generator=g)
    V = torch.empty((iters + 1, dim), dtype=torch.float64, device="cuda")
    V[0] = v / torch.linalg.vector_norm(v)
    al, be = [], []
    for j in range(iters):
        w = mv(V[j])
        for p in range(2):
            h = V[: j + 1] @ w
            w -= V[: j + 1].T @ h
            if p == 0:
                al.append(float(h[j]))
            else:
                al[-1] += float(h[j])
        b = float(torch.linalg.vector_norm(w))
        if (j + 1) % 10 == 0 or b < 1e-12:                         # the residual bound, every 10 steps
            T = np.diag(al) + np.diag(be, 1) + np.diag(be, -1)
            th, Z = np.linalg.eigh(T)
            if b * abs(Z[-1, 0]) <= tol * abs(th[0]) or b < 1e-12:
                return th[0]
        be.append(b)
        V[j + 1] = w / b
    raise AssertionError("FP64 Lanczos did not converge")


def test_fp64_central_differences(cih):
    """Central differences in FP64 at the differentiation configuration.  H
    is linear in each table entry: dH/dt_k is the fill of a table holding
    only t_k = 1 (orbital energies 0), whose values are exactly 0 or +-1.  So
    E0(H +- h dH/dt_k) can be taken in FP64 with no FP32 rounding of the
    perturbed matrix, and (E0(+h) - E0(-h)) / 2h meets the adjoint (at the
    stored matrix, Hellmann-Feynman) within the truncation h^2/6 |E'''|
    (< 1e-6 at h = 2^-10 for gaps above ~1 MeV) plus the FP64 Lanczos error
    (residual bound 1e-9 |E0|: eigenvalue error ~ (1e-7)^2 / gap, negligible
    after dividing by 2h).  Entries: the 4 largest |g| and 4 random ones."""
    B = cih.Basis(*SP)
    t = synth.tbme_table(B.tbme_len, 0)
    rowptr, col, val, nnz = cih.build_hamiltonian(B, torch.from_numpy(t).cuda())
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=1, max_iter=500, tol=1e-11)
    assert conv
    g = B.tbme_grad(rowptr, psi)[0].cpu().numpy()
    rows = torch.repeat_interleave(torch.arange(B.dim, device="cuda"), rowptr[1:] - rowptr[:-1])
    c = col.long()
    v = val[0].double()
    diag = rowptr[:-1]
    rng = np.random.default_rng(5)
    idx = np.concatenate([np.argsort(-np.abs(g))[:4], rng.choice(B.tbme_len, size=4, replace=False)])
    h = 2.0 ** -10
    e_sp0 = torch.zeros(sum(B.n_orb), dtype=torch.float64, device="cuda")
    for k in idx:
        Tk = torch.zeros((1, B.tbme_len), dtype=torch.float32, device="cuda")
        Tk[0, k] = 1.0
        ck, vk = B.fill(rowptr, nnz, Tk, e_sp=e_sp0)
        assert torch.equal(ck, col)
        vk = vk[0].double()
        assert set(torch.unique(vk).tolist()) <= {-1.0, 0.0, 1.0}
        ep = _fp64_lowest(rows, c, v + h * vk, (v + h * vk)[diag], B.dim, 3)
        em = _fp64_lowest(rows, c, v - h * vk, (v - h * vk)[diag], B.dim, 3)
        fd = (ep - em) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-6 * abs(g[k]), (int(k), fd, g[k])
    del rows, c, v
    torch.cuda.empty_cache()
