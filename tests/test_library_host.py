"""CPU checks of libcih: the shared library loads and exports every entry point
include/cih.h declares, and its host-side logic (basis, sub-determinant order,
partner ranges, two-body table layout, tridiagonal eigensolver) matches the
oracle and LAPACK.  No GPU is touched here."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cih():
    from paper_1412_5989_gb300 import build
    build.build()
    from paper_1412_5989_gb300 import cih as mod
    return mod


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cih.h")).read()
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(cih_\w+)\s*\(", src, flags=re.M)))


def test_exports_every_declared_symbol(cih):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(cih.lib, n), n
    assert set(names) == set(cih.EXPORTED)


SPACES = [(2, 2, 2, 0), (3, 3, 2, 0), (1, 1, 2, 0), (2, 0, 2, 0), (0, 2, 2, 0), (2, 1, 3, 1),
          (3, 3, 2, 8), (4, 4, 4, 0), (5, 6, 4, 1), (3, 3, 6, 0), (1, 0, 3, 1), (2, 2, 0, 0)]


@pytest.mark.parametrize("sp", SPACES)
def test_host_basis_matches_oracle(cih, sp):
    Z, N, Nmax, twoM = sp
    B = cih.Basis(Z, N, Nmax, twoM, host_only=True)
    S = oracle.Space(Z, N, Nmax, twoM)
    assert B.dim == S.dim
    assert B.n_orb == S.norb
    assert B.n_sd == S.nsd
    assert B.chan_len == S.chan_len
    t = B.tables()
    orbs = np.concatenate([S.orbitals(0), S.orbitals(1)])
    np.testing.assert_array_equal(t["orbitals"], orbs)
    for s, key in ((0, "bits_p"), (1, "bits_n")):
        w, _, _ = S.subdets(s)
        np.testing.assert_array_equal(t[key], w[:, :4])
        assert np.all(w[:, 4:] == 0)
    nb, nc, base = S.partner_ranges()
    np.testing.assert_array_equal(t["nbeg"], nb)
    np.testing.assert_array_equal(t["ncnt"], nc)
    np.testing.assert_array_equal(t["rowbase"], base)


@pytest.mark.parametrize("sp", [(2, 2, 2, 0), (3, 3, 2, 0), (4, 4, 4, 0), (5, 6, 4, 1)])
def test_table_index_matches_oracle(cih, sp):
    B = cih.Basis(*sp, host_only=True)
    S = oracle.Space(*sp)
    ntot = sum(S.norb)
    rng = np.random.default_rng(3)
    # all channel pairs against each other inside random groups, plus random quadruples
    for c in range(3):
        pa, pb, g = S.channel_pairs(c)
        if len(pa) == 0:
            continue
        for _ in range(300):
            u, v = rng.integers(len(pa), size=2)
            for (a, b_, c_, d) in ((pa[u], pb[u], pa[v], pb[v]), (pb[u], pa[u], pa[v], pb[v]),
                                   (pa[v], pb[v], pb[u], pa[u])):
                assert B.tbme_index(int(a), int(b_), int(c_), int(d)) == S.tbme_index(int(a), int(b_), int(c_), int(d))
    for _ in range(2000):
        a, b_, c_, d = (int(x) for x in rng.integers(ntot, size=4))
        assert B.tbme_index(a, b_, c_, d) == S.tbme_index(a, b_, c_, d)


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (2, 1, 3, 1), (4, 4, 4, 0), (1, 0, 3, 1), (0, 2, 2, 0)])
def test_onebody_layout_matches_oracle(cih, sp):
    """The library's one-body table layout gives every orbital pair the
    oracle's index (its own construction: a stable sort by (species, 2m,
    parity) instead of the oracle's scans)."""
    B = cih.Basis(*sp, host_only=True)
    S = oracle.Space(*sp)
    assert B.onebody_len == S.onebody_len
    n = sum(B.n_orb)
    for a in range(n):
        for c in range(n):
            assert B.onebody_index(a, c) == S.onebody_index(a, c), (a, c)
    assert B.onebody_index(-1, 0) == -1 and B.onebody_index(0, n) == -1


def test_empty_space(cih):
    B = cih.Basis(2, 2, 2, 1, host_only=True)       # even A, odd 2M
    assert B.dim == 0


def test_bad_arguments_raise(cih):
    with pytest.raises(cih.CihError):
        cih.Basis(-1, 2, 2, 0, host_only=True)
    with pytest.raises(cih.CihError):
        cih.Basis(2, 2, -1, 0, host_only=True)
    # more than 256 orbitals per species
    with pytest.raises(cih.CihError) as e:
        cih.Basis(2, 2, 8, 0, host_only=True)
    assert e.value.code == -5


def test_tridiagonal_eigensolver(cih):
    rng = np.random.default_rng(0)
    for n in (1, 2, 3, 10, 60, 200):
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
        w, Z = cih.tridiag_eigen(d, e)
        np.testing.assert_allclose(w, np.linalg.eigvalsh(T), rtol=0, atol=1e-12 * max(1, np.abs(w).max()))
        np.testing.assert_allclose(T @ Z, Z * w, rtol=0, atol=1e-11)
        np.testing.assert_allclose(Z.T @ Z, np.eye(n), rtol=0, atol=1e-12)
    # graded and degenerate cases: the 1-D Laplacian and a zero off-diagonal
    n = 40
    w, _ = cih.tridiag_eigen(np.full(n, 2.0), np.full(n - 1, -1.0))
    np.testing.assert_allclose(w, 2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)), atol=1e-13)
    w, Z = cih.tridiag_eigen(np.array([3.0, 1.0, 2.0]), np.zeros(2))
    assert w.tolist() == [1.0, 2.0, 3.0]


def test_entry_points_reject_bad_arguments_without_a_gpu(cih):
    """Argument checks of the device entry points run before any device work:
    a host-only handle, NULL arrays, K, nev or budget out of range."""
    import ctypes as C
    lib = cih.lib
    B = cih.Basis(3, 3, 2, 0, host_only=True)
    h = B._h
    assert lib.cih_tbme_interleave(0, 10, None, None, None) == -1
    assert lib.cih_tbme_interleave(4, -1, None, None, None) == -1
    assert lib.cih_set_launch(h, 12, 0) == -1
    assert lib.cih_set_launch(h, 16, 33) == -1
    assert lib.cih_set_launch(None, 16, 0) == -1
    assert lib.cih_set_launch(h, 8, 2) == 0 and lib.cih_set_launch(h, 16, 0) == 0
    assert lib.cih_set_count_mode(h, 2) == -1 and lib.cih_set_count_mode(None, 0) == -1
    assert lib.cih_set_count_mode(h, 1) == 0 and lib.cih_set_count_mode(h, 0) == 0
    rc = C.c_int32()
    # device calls refuse a host-only handle
    assert lib.cih_ham_count(h, C.c_void_p(16), None, None) == -1
    assert lib.cih_ham_fill(h, C.c_void_p(16), 1, 20.0, C.c_void_p(16), None, C.c_void_p(16), C.c_void_p(16), None) == -1
    assert lib.cih_ham_fill_batched(h, C.c_void_p(16), 4, 20.0, C.c_void_p(16), None, C.c_void_p(16),
                                    C.c_void_p(16), None) == -1
    ev = (C.c_double * 4)()
    assert lib.cih_lanczos_lowest_em(h, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 1, 1, 10, 1e-8, ev,
                                     None, None) == -1
    assert lib.cih_ham_spmv(h, C.c_void_p(16), C.c_void_p(16), C.c_void_p(16), 1, 0, C.c_void_p(16),
                            C.c_void_p(24), None) == -1
    f2 = C.c_double()
    assert lib.cih_ham_upper_sumsq(h, C.c_void_p(16), 0, 1, C.c_void_p(16), 1, 0, C.byref(f2), None) == -1
    noop = lib.cih_lanczos_lowest_shard.argtypes[14](lambda ctx: 0)
    assert lib.cih_lanczos_lowest_shard(h, C.c_void_p(16), 0, 1, C.c_void_p(16), C.c_void_p(16), 1, 0, 1, 10,
                                        1e-8, 1.0, C.c_void_p(16), C.c_void_p(24), noop, None, ev, None,
                                        None) == -1
    w, c, ms = C.c_int32(), C.c_int32(), C.c_float()
    assert lib.cih_autotune_fill(h, C.c_void_p(16), 1, 20.0, C.c_void_p(16), 0, None, C.c_void_p(16),
                                 C.c_void_p(16), None, C.byref(w), C.byref(c), C.byref(ms)) == -1
    # batch: empty batch is a no-op, negative count, bad nev / budget, host-only instance
    assert lib.cih_batch_solve(None, 0, 20.0, 5, 100, 1e-8, 0, None) == 0
    assert lib.cih_batch_solve(None, -1, 20.0, 5, 100, 1e-8, 0, None) == -1
    inst = (cih.Instance * 1)()
    inst[0] = cih.Instance(h, 1, None, None, ev, None, 0, 0, -1, 0)
    assert lib.cih_batch_solve(inst, 1, 20.0, 0, 100, 1e-8, 0, None) == -1
    assert lib.cih_batch_solve(inst, 1, 20.0, 1, 100, 1e-8, -5, None) == -1
    assert lib.cih_batch_solve(inst, 1, 20.0, 1, 100, 1e-8, 0, None) == -1     # host-only basis
    assert lib.cih_batch_solve(inst, 300, 20.0, 1, 100, 1e-8, 0, None) == -5   # too many instances
    B.close()
