"""GPU: every value layout of the fill on small spaces, for set counts that
take each code path: K = 1, 3 (no float4 reads), 4, 5, 8, 16 and 20 (lanes over
sets from 16 on, 20/4 = 5 lanes per element, which does not divide 32, so
the per-lane writes), with and without a one-body override; the three layouts bit-identical to
each other and the whole matrix of the first and last set against the
oracle."""
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


def within(v, ref):
    v = np.asarray(v, dtype=np.float64)
    return np.all(np.abs(v - ref) <= 1e-5 * (np.abs(ref) + 1.0))


@pytest.mark.parametrize("sp", [(3, 3, 4, 0), (2, 1, 3, 1)])
@pytest.mark.parametrize("K", [1, 3, 4, 5, 8, 16, 20])
@pytest.mark.parametrize("override", [False, True])
def test_layouts_against_oracle(cih, sp, K, override):
    B = cih.Basis(*sp)
    S = oracle.Space(*sp)
    T = synth.tbme_tables(B.tbme_len, range(50, 50 + K))
    esp = synth.single_particle_energies(sum(B.n_orb), 3) if override else None
    Tt = torch.from_numpy(T).cuda()
    esp_t = torch.from_numpy(esp) if override else None
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, Tt, e_sp=esp_t)                   # set-major
    til = cih.tbme_interleave(Tt)
    col2, val2 = B.fill_interleaved(rowptr, nnz, til, K, e_sp=esp_t)
    col3, vem = B.fill_batched(rowptr, nnz, til, K, e_sp=esp_t)      # element-major
    B.check()
    assert torch.equal(col2, col) and torch.equal(col3, col)
    assert torch.equal(val2, val)
    assert torch.equal(vem.t(), val)
    c = col.cpu().numpy()
    for k in sorted({0, K - 1}):                                     # first and last set
        rp_o, col_o, val_o = S.half_csr(T[k], esp)
        np.testing.assert_array_equal(rowptr.cpu().numpy(), rp_o)
        np.testing.assert_array_equal(c, col_o)
        assert within(val[k].cpu().numpy(), val_o), k


def test_batch_with_a_repeated_basis_and_two_sets(cih):
    """The same basis twice in one batch (its count scans then run one after
    the other) and a two-set instance: eigenvalues as the step-by-step calls."""
    B = cih.Basis(3, 3, 2, 0)
    t0 = torch.from_numpy(synth.tbme_table(B.tbme_len, 7)).cuda().unsqueeze(0)
    t2 = torch.from_numpy(synth.tbme_tables(B.tbme_len, [8, 9])).cuda()
    rc, out = cih.solve_batch([(B, t0), (B, t2)], nev=3, max_iter=300, tol=1e-10)
    assert rc == 0 and [o["wave"] for o in out] == [0, 0]
    for t, o in ((t0, out[0]), (t2, out[1])):
        rowptr, col, val, nnz = cih.build_hamiltonian(B, t)
        ev, psi, conv = B.lanczos(rowptr, col, val, nev=3, max_iter=300, tol=1e-10)
        assert conv
        np.testing.assert_array_equal(ev, o["evals"])
        assert torch.equal(B.tbme_grad(rowptr, psi), o["grad"])


@pytest.mark.parametrize("K", [1, 3])
@pytest.mark.parametrize("pinned", [True, False])
def test_build_to_host_matches_device_fill(cih, K, pinned):
    """Host tables in, host matrix out (chunked fill with overlapped copies):
    identical to the device-resident count + fill; a too small capacity is
    refused with the count reported."""
    sp = (3, 3, 4, 0)
    B = cih.Basis(*sp)
    T = synth.tbme_tables(B.tbme_len, range(20, 20 + K))
    esp = synth.single_particle_energies(sum(B.n_orb), 5)
    rowptr, nnz = B.count()
    col, val = B.fill(rowptr, nnz, torch.from_numpy(T).cuda(), e_sp=torch.from_numpy(esp))
    cap = nnz + 17
    rp_h = torch.zeros(B.dim + 1, dtype=torch.int64, pin_memory=pinned)
    col_h = torch.zeros(cap, dtype=torch.int32, pin_memory=pinned)
    val_h = torch.zeros((K, cap), dtype=torch.float32, pin_memory=pinned)
    tb_h = torch.from_numpy(T)
    if pinned:
        tb_h = tb_h.pin_memory()
    n = B.build_to_host(tb_h, rp_h, col_h, val_h, e_sp=esp)
    B.check()
    assert n == nnz
    assert torch.equal(rp_h, rowptr.cpu())
    assert torch.equal(col_h[:nnz], col.cpu())
    assert torch.equal(val_h[:, :nnz], val.cpu())
    small = torch.zeros(nnz - 1, dtype=torch.int32)
    with pytest.raises(cih.CihError) as e:
        B.build_to_host(tb_h, rp_h, small, torch.zeros((K, nnz - 1), dtype=torch.float32))
    assert e.value.code == -3
