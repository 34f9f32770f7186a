"""GPU: d(lowest eigenvalue)/d(two-body table) at 4+4 Nmax=4, 2M=0, one table.

The adjoint (Hellmann-Feynman: g_t = sum over stored elements using t of
w * phase * psi_i psi_j) through torch.autograd, against

- central finite differences of the lowest eigenvalue on 32 random table
  entries, the 64 perturbed tables built and solved as one batch of K = 64
  sets sharing the structure;
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
    assert float(e0) == ev[0][0]
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
