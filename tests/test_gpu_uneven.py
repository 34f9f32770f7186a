"""GPU: the uneven batch (3+3 Nmax=6, 4+4 Nmax=6, 5+6 Nmax=4 2M=1; one table
each, seeds 100-102) through the fused count -> admission -> fill -> Lanczos ->
adjoint call.

- nonzero counts equal the independently sized counts (generating-function
  sizing of the basis and the selection rules);
- eigenvalues and gradients are bit-identical to the same steps called one by
  one (every step is deterministic);
- one instance's eigenvalues agree with the oracle's Lanczos on the same
  stored matrix, its gradient with the oracle's adjoint on the same vector;
- a budget that holds one instance at a time runs them in successive waves
  with the same results; a budget below every instance admits none.
"""
import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPACES = [(3, 3, 6, 0), (4, 4, 6, 0), (5, 6, 4, 1)]
SEEDS = [100, 101, 102]
HALF_NNZ = [60_236_339, 924_863_410, 207_049_448]
NEV, ITERS, TOL = 5, 400, 1e-9


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.fixture(scope="module")
def batch(cih):
    bases = [cih.Basis(*sp) for sp in SPACES]
    tabs = [torch.from_numpy(synth.tbme_table(B.tbme_len, s)).cuda().unsqueeze(0) for B, s in zip(bases, SEEDS)]
    rc, out = cih.solve_batch(list(zip(bases, tabs)), nev=NEV, max_iter=ITERS, tol=TOL)
    yield bases, tabs, rc, out
    torch.cuda.empty_cache()


def test_counts_and_status(cih, batch):
    bases, tabs, rc, out = batch
    assert rc == 0
    for o, n in zip(out, HALF_NNZ):
        assert o["status"] == 0 and o["wave"] == 0
        assert o["nnz"] == n
        assert o["bytes"] > 8 * n


def test_fused_equals_step_by_step(cih, batch):
    bases, tabs, rc, out = batch
    for B, t, o in zip(bases, tabs, out):
        rowptr, col, val, nnz = cih.build_hamiltonian(B, t)
        assert nnz == o["nnz"]
        ev, psi, conv = B.lanczos(rowptr, col, val, nev=NEV, max_iter=ITERS, tol=TOL)
        assert conv
        np.testing.assert_array_equal(ev, o["evals"])
        del col, val
        g = B.tbme_grad(rowptr, psi)
        assert torch.equal(g, o["grad"])
        del psi, g
        torch.cuda.empty_cache()


def test_one_instance_against_oracle(cih, batch):
    bases, tabs, rc, out = batch
    B, t, o = bases[0], tabs[0], out[0]
    rowptr, col, val, nnz = cih.build_hamiltonian(B, t)
    ev_o, _, _, conv_o = oracle.lanczos(rowptr.cpu().numpy(), col.cpu().numpy(), val[0].cpu().numpy(),
                                        nev=NEV, max_iter=ITERS, tol=1e-12)
    assert conv_o
    np.testing.assert_allclose(o["evals"][0], ev_o, rtol=1e-5)
    ev, psi, conv = B.lanczos(rowptr, col, val, nev=1, max_iter=ITERS, tol=TOL)
    S = oracle.Space(*SPACES[0])
    g_o = S.grad_elementwise(rowptr.cpu().numpy(), col.cpu().numpy(), psi[0].cpu().numpy())
    g = B.tbme_grad(rowptr, psi)[0].cpu().numpy()
    np.testing.assert_allclose(g, g_o, rtol=0, atol=1e-9)


def test_admission_waves(cih, batch):
    bases, tabs, rc, out = batch
    rowptr_bytes = sum(8 * (B.dim + 1) for B in bases)
    budget = rowptr_bytes + max(o["bytes"] for o in out) + (1 << 20)
    rc2, out2 = cih.solve_batch(list(zip(bases, tabs)), nev=NEV, max_iter=ITERS, tol=TOL, hbm_budget=budget)
    assert rc2 == 0
    waves = [o["wave"] for o in out2]
    assert waves[0] == 0 and all(b >= a for a, b in zip(waves, waves[1:])) and waves[-1] >= 1
    for a, b in zip(out, out2):
        np.testing.assert_array_equal(a["evals"], b["evals"])
        assert torch.equal(a["grad"], b["grad"])
    rc3, out3 = cih.solve_batch(list(zip(bases, tabs)), nev=NEV, max_iter=ITERS, tol=TOL,
                                hbm_budget=rowptr_bytes + (1 << 20))
    assert rc3 == 1
    assert all(o["status"] == -3 and o["wave"] == -1 for o in out3)
    assert all(np.isnan(o["evals"]).all() for o in out3)
