"""Pins of the CPU oracle to facts other than itself (closed forms, brute force,
hand-derived fixtures, library routines).  CPU only.

Each pin is chosen so that a plausible mistake in the oracle -- a dropped term,
a wrong sign or index, a transposed operand, a wrong truncation -- fails one:
  * orbital shells hold (N+1)(N+2) states (closed form);
  * basis dimensions equal an independent generating-function count and, on
    tiny cases, a brute-force enumeration of all determinants;
  * the Slater-Condon matrix equals the ket-driven application of every
    operator term (signs, indices, spectator sums);
  * zero / unit-diagonal / two-particle tables give closed-form matrices;
  * the Jacobi and bisection eigensolvers match numpy's LAPACK routines;
  * Lanczos matches the dense solve; the gradient matches central finite
    differences, the brute-force two-body density and the Euler identity.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1412_5989_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def shell_orbitals(Nmax_shell):
    """(N, l, 2j, 2m) in the documented order, from the oscillator closed form."""
    out = []
    for N in range(Nmax_shell + 1):
        for l in range(N % 2, N + 1, 2):
            for j2 in (2 * l - 1, 2 * l + 1):
                if j2 < 0:
                    continue
                for m2 in range(-j2, j2 + 1, 2):
                    out.append((N, l, j2, m2))
    return out


# ---------------------------------------------------------------- orbitals

@pytest.mark.parametrize("Z,N,Nmax,norb", [(3, 3, 2, 40), (4, 4, 4, 112), (4, 4, 6, 240), (5, 6, 4, 112)])
def test_orbital_counts(Z, N, Nmax, norb):
    S = oracle.Space(Z, N, Nmax, (Z + N) % 2)
    assert S.norb == (norb, norb)
    o = S.orbitals(0)
    for sh in range(o[:, 0].max() + 1):
        assert (o[:, 0] == sh).sum() == (sh + 1) * (sh + 2)
    # j = l +- 1/2, l = N mod 2, |m| <= j, strictly ascending (N, l, 2j, 2m)
    assert np.all(np.abs(o[:, 2] - 2 * o[:, 1]) == 1)
    assert np.all(o[:, 1] % 2 == o[:, 0] % 2)
    assert np.all(np.abs(o[:, 3]) <= o[:, 2])
    keys = [tuple(r) for r in o]
    assert keys == sorted(set(keys))
    assert keys == shell_orbitals(o[:, 0].max())


# ---------------------------------------------------------------- dimensions

def dim_generating_function(Z, N, Nmax, twoM):
    """Independent count of the M-scheme dimension: per species, a DP over the
    orbitals of the number of k-subsets by (sum N, sum 2m); then pair them."""
    def lowest(k):
        left, sh, s, top = k, 0, 0, -1
        while left > 0:
            put = min(left, (sh + 1) * (sh + 2))
            s += put * sh
            left -= put
            top = sh
            sh += 1
        return s, top

    (n0p, nfp), (n0n, nfn) = lowest(Z), lowest(N)
    Nlim = n0p + n0n + Nmax

    def table(k, nf):
        if k == 0:
            return {(0, 0): 1}
        orbs = shell_orbitals(nf + Nmax)
        # dp[c][(Nsum, Msum)] = number of c-subsets of the orbitals seen so far
        dp = [dict() for _ in range(k + 1)]
        dp[0][(0, 0)] = 1
        for (n, _, _, m) in orbs:
            for c in range(k - 1, -1, -1):
                for (Ns, Ms), v in list(dp[c].items()):
                    if Ns + n <= Nlim:
                        key = (Ns + n, Ms + m)
                        dp[c + 1][key] = dp[c + 1].get(key, 0) + v
        return dp[k]

    tp, tn = table(Z, nfp), table(N, nfn)
    dim = 0
    for (Np_, Mp), a in tp.items():
        for (Nn_, Mn), b in tn.items():
            Nt = Np_ + Nn_
            if Mp + Mn == twoM and Nt <= Nlim and (Nlim - Nt) % 2 == 0:
                dim += a * b
    return dim


@pytest.mark.parametrize("Z,N,Nmax,twoM,dim", [
    (2, 2, 2, 0, 59), (3, 3, 2, 0, 800), (4, 4, 4, 0, 143792), (3, 3, 6, 0, 197822),
    (5, 6, 4, 1, 814092), (1, 1, 2, 0, 24), (2, 0, 2, 0, 12), (4, 4, 6, 0, 2217754)])
def test_dimension(Z, N, Nmax, twoM, dim):
    S = oracle.Space(Z, N, Nmax, twoM)
    assert S.dim == dim
    if Nmax <= 4:
        assert dim_generating_function(Z, N, Nmax, twoM) == dim


def test_odd_M_even_A_is_empty():
    S = oracle.Space(2, 2, 2, 1)
    assert S.dim == 0


def occupations(S):
    """Combined occupation sets of every basis state, via the sub-det bit strings."""
    wp, _, _ = S.subdets(0)
    wn, _, _ = S.subdets(1)

    def bits(w, n):
        return [a for a in range(n) if (int(w[a >> 6]) >> (a & 63)) & 1]

    out = []
    for i in range(S.dim):
        p, n = S.basis_state(i)
        out.append(tuple(bits(wp[p], S.norb[0]) + [S.norb[0] + b for b in bits(wn[n], S.norb[1])]))
    return out


@pytest.mark.parametrize("Z,N,Nmax", [(2, 2, 2), (1, 2, 2), (2, 1, 3)])
def test_basis_brute_force(Z, N, Nmax):
    """All determinants of the combined orbitals, filtered by the definition;
    the oracle's basis must be exactly this set, ordered by (proton sub-det
    key, neutron sub-det key) with key (2M, N mod 2, N, bit string)."""
    twoM = (Z + N) % 2
    S = oracle.Space(Z, N, Nmax, twoM)
    op, on = S.orbitals(0), S.orbitals(1)
    (n0p, _), (n0n, _) = [(sum(sorted(o[:, 0])[:k]), 0) for o, k in ((op, Z), (on, N))]
    Nlim = n0p + n0n + Nmax
    states = []
    for P in itertools.combinations(range(len(op)), Z):
        for Q in itertools.combinations(range(len(on)), N):
            Nt = sum(op[a, 0] for a in P) + sum(on[b, 0] for b in Q)
            Mt = sum(op[a, 3] for a in P) + sum(on[b, 3] for b in Q)
            if Mt == twoM and Nt <= Nlim and (Nlim - Nt) % 2 == 0:
                states.append((P, Q))

    def key(o, T):
        Nsum = sum(o[a, 0] for a in T)
        return (sum(o[a, 3] for a in T), Nsum % 2, Nsum, sum(1 << a for a in T))

    states.sort(key=lambda s: (key(op, s[0]), key(on, s[1])))
    expect = [tuple(list(P) + [len(op) + b for b in Q]) for P, Q in states]
    assert occupations(S) == expect


def test_partner_ranges_contiguous():
    S = oracle.Space(3, 3, 2, 0)
    _, Np, Mp = S.subdets(0)
    _, Nn, Mn = S.subdets(1)
    nb, nc, base = S.partner_ranges()
    Nlim = 2 + 2
    for p in range(S.nsd[0]):
        ok = [(Mp[p] + Mn[k] == 0 and Np[p] + Nn[k] <= Nlim and (Nlim - Np[p] - Nn[k]) % 2 == 0)
              for k in range(S.nsd[1])]
        idx = np.nonzero(ok)[0]
        assert len(idx) == nc[p] > 0
        assert idx[0] == nb[p] and idx[-1] == nb[p] + nc[p] - 1
    assert base[-1] == S.dim


# ---------------------------------------------------------------- table layout

def test_table_sizes_and_pair_limits():
    # 3+3 Nmax2: pair quanta limits pp/nn 3, pn 4
    S = oracle.Space(3, 3, 2, 0)
    o = np.concatenate([S.orbitals(0), S.orbitals(1)])
    for c, lim in ((0, 3), (1, 3), (2, 4)):
        pa, pb, g = S.channel_pairs(c)
        assert np.all(o[pa, 0] + o[pb, 0] <= lim)
        assert np.all(pa < pb)
        # every orbital pair of the channel under the limit is present
        if c == 0:
            want = [(a, b) for a in range(40) for b in range(a + 1, 40) if o[a, 0] + o[b, 0] <= lim]
        elif c == 1:
            want = [(a, b) for a in range(40, 80) for b in range(a + 1, 80) if o[a, 0] + o[b, 0] <= lim]
        else:
            want = [(a, b) for a in range(40) for b in range(40, 80) if o[a, 0] + o[b, 0] <= lim]
        assert sorted(zip(pa.tolist(), pb.tolist())) == sorted(want)
        # groups ascending by (2M_pair, parity), lexicographic inside
        keys = [(o[a, 3] + o[b, 3], (o[a, 0] + o[b, 0]) % 2, a, b) for a, b in zip(pa, pb)]
        assert keys == sorted(keys)
        sizes = np.bincount(g)
        assert S.chan_len[c] == int(sum(n * (n + 1) // 2 for n in sizes))
    # table bytes quoted for the benchmark workloads
    assert oracle.Space(4, 4, 4, 0).tbme_len * 4 == pytest.approx(2.2e6, rel=0.01)
    assert oracle.Space(4, 4, 6, 0).tbme_len * 4 == pytest.approx(19.9e6, rel=0.01)


def test_table_index_symmetries():
    S = oracle.Space(2, 2, 2, 0)
    pa, pb, g = S.channel_pairs(2)
    rng = np.random.default_rng(0)
    for _ in range(200):
        u, v = rng.integers(len(pa), size=2)
        if g[u] != g[v]:
            assert S.tbme_index(pa[u], pb[u], pa[v], pb[v])[0] == -1
            continue
        i1, s1 = S.tbme_index(pa[u], pb[u], pa[v], pb[v])
        i2, s2 = S.tbme_index(pa[v], pb[v], pa[u], pb[u])      # Hermitian partner
        i3, s3 = S.tbme_index(pb[u], pa[u], pa[v], pb[v])      # swapped bra pair
        i4, s4 = S.tbme_index(pb[u], pa[u], pb[v], pa[v])      # both swapped
        assert i1 == i2 == i3 == i4 >= 0
        assert (s1, s2, s3, s4) == (1, 1, -1, 1)


# ---------------------------------------------------------------- golden fixtures

@pytest.mark.parametrize("name", ["two_nucleon_0s.json", "alpha_0s.json"])
def test_golden(name):
    d = json.load(open(os.path.join(GOLDEN, name)))
    sp = d["space"]
    S = oracle.Space(sp["Z"], sp["N"], sp["Nmax"], sp["twoM"])
    assert S.dim == d["dim"] and S.tbme_len == len(d["tbme"])
    t = np.array(d["tbme"], dtype=np.float32)
    H = S.dense_sc(t, hw=sp["hbar_omega"])
    np.testing.assert_allclose(H, np.array(d["H"]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.jacobi(H), d["eigenvalues"], rtol=1e-13)


# ---------------------------------------------------------------- matrix elements

@pytest.mark.parametrize("Z,N,Nmax,twoM", [(2, 2, 2, 0), (3, 3, 2, 0), (2, 1, 2, 1), (3, 0, 2, 1),
                                            (2, 2, 2, 4), (2, 1, 2, 5), (1, 2, 3, 7), (2, 2, 3, 8),
                                            (3, 3, 2, 6), (3, 3, 2, 8)])
def test_slater_condon_equals_operator_application(Z, N, Nmax, twoM):
    # large 2M puts the highest-m orbitals in play as spectators
    S = oracle.Space(Z, N, Nmax, twoM)
    assert S.dim > 0
    t = synth.tbme_table(S.tbme_len, 7)
    esp = synth.single_particle_energies(S.norb[0] + S.norb[1], 3)
    Hb = S.dense_brute(t, esp)
    Hs = S.dense_sc(t, esp)
    np.testing.assert_allclose(Hs, Hb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Hb, Hb.T, rtol=0, atol=1e-12)   # Hermiticity


def test_known_nnz_and_structure():
    for (Z, N, Nmax, full, half) in [(2, 2, 2, 1691, 875), (3, 3, 2, 69152, 34976)]:
        S = oracle.Space(Z, N, Nmax, 0)
        t = synth.tbme_table(S.tbme_len, 1)
        H = S.dense_sc(t)
        occ = occupations(S)
        # structure: <= 2 particles moved  <=> |symmetric difference| <= 4
        mask = np.array([[len(set(a) ^ set(b)) <= 4 for b in occ] for a in occ])
        assert mask.sum() == full
        assert np.all(H[~mask] == 0)
        rp, col, val = S.half_csr(t)
        assert rp[-1] == half == (full + S.dim) // 2
        for i in range(S.dim):
            cols = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(cols) > 0) and cols[0] == i
            assert np.array_equal(cols, np.nonzero(mask[i, i:])[0] + i)
            np.testing.assert_array_equal(val[rp[i]:rp[i + 1]], H[i, cols].astype(np.float32))


def test_zero_tbme_spectrum_closed_form():
    S = oracle.Space(3, 3, 2, 0)
    H = S.dense_sc(np.zeros(S.tbme_len, np.float32))
    assert np.count_nonzero(H - np.diag(np.diag(H))) == 0
    vals, counts = np.unique(np.diag(H), return_counts=True)
    # hbar_omega * sum_a (N_a + 3/2) over 6 nucleons with N_tot = 2 or 4
    assert vals.tolist() == [220.0, 260.0] and counts.tolist() == [10, 790]


def test_one_body_override_gives_sorted_diagonal():
    S = oracle.Space(2, 2, 2, 0)
    esp = synth.single_particle_energies(S.norb[0] + S.norb[1], 11)
    H = S.dense_sc(np.zeros(S.tbme_len, np.float32), esp)
    occ = occupations(S)
    want = np.array([sum(esp[a] for a in o) for o in occ])
    np.testing.assert_allclose(np.diag(H), want, rtol=1e-14)
    np.testing.assert_allclose(oracle.jacobi(H), np.sort(want), rtol=1e-13)


def test_unit_diagonal_table_counts_pairs():
    for (Z, N) in [(3, 3), (2, 1), (3, 0)]:
        S = oracle.Space(Z, N, 2, (Z + N) % 2)
        t = np.zeros(S.tbme_len, np.float32)
        for c in range(3):
            pa, pb, g = S.channel_pairs(c)
            for a, b in zip(pa, pb):
                idx, s = S.tbme_index(a, b, a, b)
                t[idx] = 1.0
        H = S.dense_sc(t)
        H0 = S.dense_sc(np.zeros_like(t))
        A = Z + N
        np.testing.assert_array_equal(H - H0, np.eye(S.dim) * (A * (A - 1) / 2))


@pytest.mark.parametrize("Z,N", [(1, 1), (2, 0), (0, 2)])
def test_two_particle_system(Z, N):
    """H on two particles = e_a + e_b on the diagonal plus the table block."""
    S = oracle.Space(Z, N, 2, 0)
    t = synth.tbme_table(S.tbme_len, 5)
    H = S.dense_sc(t)
    occ = occupations(S)
    o = np.concatenate([S.orbitals(0), S.orbitals(1)])
    c = 2 if Z == 1 else (0 if Z == 2 else 1)
    pa, pb, g = S.channel_pairs(c)
    pairs = list(zip(pa.tolist(), pb.tolist()))
    # packed upper triangle of each group, written out here
    start = {}
    for k, gg in enumerate(g):
        start.setdefault(gg, k)
    sizes = np.bincount(g)
    goff = np.concatenate([[0], np.cumsum(sizes * (sizes + 1) // 2)])
    chan_base = sum(S.chan_len[:c])
    for i, oi in enumerate(occ):
        for j, oj in enumerate(occ):
            ki, kj = pairs.index(oi), pairs.index(oj)
            if g[ki] != g[kj]:
                assert H[i, j] == 0
                continue
            u, v = sorted((ki - start[g[ki]], kj - start[g[kj]]))
            n = sizes[g[ki]]
            want = t[chan_base + goff[g[ki]] + u * n - u * (u - 1) // 2 + (v - u)]
            if i == j:
                want = want + 20.0 * (o[oi[0], 0] + 1.5) + 20.0 * (o[oi[1], 0] + 1.5)
            assert H[i, j] == pytest.approx(float(want), abs=1e-12)


# ---------------------------------------------------------------- eigensolvers

def test_jacobi_against_lapack():
    rng = np.random.default_rng(2)
    for n in (1, 2, 7, 40):
        A = rng.standard_normal((n, n))
        A = A + A.T
        w, V = oracle.jacobi(A, vectors=True)
        np.testing.assert_allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-11)
        np.testing.assert_allclose(A @ V, V * w, rtol=0, atol=1e-10)


def test_tridiagonal_bisection():
    n = 30   # discrete Laplacian: 2 - 2 cos(k pi / (n+1))
    a, b = np.full(n, 2.0), np.full(n - 1, -1.0)
    for r in (0, 1, 5, 29):
        assert oracle.tridiag_eig(a, b, r) == pytest.approx(2 - 2 * math.cos((r + 1) * math.pi / (n + 1)), abs=1e-13)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal(50), rng.standard_normal(49)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    w = np.linalg.eigvalsh(T)
    for r in range(0, 50, 7):
        assert oracle.tridiag_eig(a, b, r) == pytest.approx(w[r], abs=1e-12)


def dense_from_half(rp, col, val):
    n = len(rp) - 1
    H = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            H[i, col[k]] = H[col[k], i] = val[k]
    return H


def test_lanczos_matches_dense():
    S = oracle.Space(3, 3, 2, 0)
    t = synth.tbme_table(S.tbme_len, 0)
    rp, col, val = S.half_csr(t)
    H = dense_from_half(rp, col, val)
    ev, vec, it, conv = oracle.lanczos(rp, col, val, nev=5, max_iter=300, tol=1e-12)
    assert conv
    w = np.linalg.eigvalsh(H)
    np.testing.assert_allclose(ev, w[:5], rtol=1e-10)
    vec = vec / np.linalg.norm(vec)
    assert np.linalg.norm(H @ vec - ev[0] * vec) <= 1e-8 * np.abs(w).max()


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (2, 1, 3, 1), (1, 0, 3, 1)])
def test_half_spmv_equals_the_dense_product(sp):
    """The half-stored product (upper triangle with diagonal, mirrored on the
    fly) against the dense Slater-Condon matrix times x: a dropped mirror term,
    a doubled diagonal or a transposed access fails it."""
    S = oracle.Space(*sp)
    t = synth.tbme_table(S.tbme_len, 4)
    rp, col, val = S.half_csr(t)
    x = np.random.default_rng(1).standard_normal(S.dim)
    H = S.dense_sc(t)
    want = dense_from_half(rp, col, val) @ x
    got = oracle.half_spmv(rp, col, val, x)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    np.testing.assert_allclose(got, H @ x, rtol=0, atol=1e-5 * np.abs(H).sum(axis=1).max() * np.abs(x).max())


def test_lanczos_degenerate_spectrum_gives_distinct_values():
    S = oracle.Space(3, 3, 2, 0)
    rp, col, val = S.half_csr(np.zeros(S.tbme_len, np.float32))
    ev, vec, it, conv = oracle.lanczos(rp, col, val, nev=2, max_iter=50, tol=1e-12)
    assert conv
    np.testing.assert_allclose(ev, [220.0, 260.0], rtol=1e-13)


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("Z,N", [(2, 2), (2, 1)])
def test_gradient(Z, N):
    S = oracle.Space(Z, N, 2, (Z + N) % 2)
    t = synth.tbme_table(S.tbme_len, 9)
    H = S.dense_sc(t)
    w, V = np.linalg.eigh(H)
    assert w[1] - w[0] > 1e-3
    psi = V[:, 0]
    rp, col, val = S.half_csr(t)
    g = S.grad_elementwise(rp, col, psi)
    # brute-force two-body density of every parameter's operator
    np.testing.assert_allclose(g, S.density_brute(psi), rtol=0, atol=1e-12)
    # Euler identity: H is linear in (e, V), so E0 = <one-body> + sum_t g_t t
    H1 = S.dense_sc(np.zeros_like(t))
    assert psi @ H1 @ psi + g @ t.astype(np.float64) == pytest.approx(w[0], abs=1e-9)
    # central finite differences in FP64 on 32 random parameters
    rng = np.random.default_rng(1)
    t64 = t.astype(np.float64)
    for k in rng.choice(S.tbme_len, size=32, replace=False):
        h = 1e-4 * max(1.0, abs(t64[k]))
        e = np.zeros_like(t64)
        e[k] = 1.0
        # H is linear in t: H(t + h e) = H(t) + h dH/dt, with dH/dt built by the
        # oracle from a table that is 1 at k and 0 elsewhere
        dH = S.dense_sc(e.astype(np.float32)) - H1
        Ep = np.linalg.eigvalsh(H + h * dH)[0]
        Em = np.linalg.eigvalsh(H - h * dH)[0]
        assert (Ep - Em) / (2 * h) == pytest.approx(g[k], abs=1e-6)


# ---------------------------------------------------------------- one-body table

def _t_full(S, t1):
    """The symmetric one-body matrix t[a, c] written out from the table
    (zero outside the one-species, equal-2m, equal-parity groups)."""
    n = S.norb[0] + S.norb[1]
    T = np.zeros((n, n))
    for a in range(n):
        for c in range(n):
            k = S.onebody_index(a, c)
            if k >= 0:
                T[a, c] = t1[k]
    return T


def test_onebody_layout_groups():
    """t_ac has an entry exactly when a and c are one species with equal 2m
    and equal N parity; the packed triangles tile the table."""
    S = oracle.Space(3, 2, 3, 1)
    o = np.concatenate([S.orbitals(0), S.orbitals(1)])
    sp = np.array([0] * S.norb[0] + [1] * S.norb[1])
    n = len(o)
    seen = set()
    for a in range(n):
        for c in range(n):
            k = S.onebody_index(a, c)
            same = sp[a] == sp[c] and o[a, 3] == o[c, 3] and (o[a, 0] - o[c, 0]) % 2 == 0
            assert (k >= 0) == same
            if same:
                assert k == S.onebody_index(c, a)
                seen.add(k)
    assert seen == set(range(S.onebody_len))


@pytest.mark.parametrize("Z,N,Nmax,twoM", [(1, 0, 3, 1), (0, 1, 4, 3), (1, 0, 4, -1)])
def test_onebody_single_particle_block(Z, N, Nmax, twoM):
    """One particle: H is the one-body matrix itself on the orbitals of the
    basis (closed form), whatever the two-body table."""
    S = oracle.Space(Z, N, Nmax, twoM)
    t1 = synth.onebody_table(S.onebody_len, 3)
    S.set_onebody(t1)
    T = _t_full(S, t1)
    orb = [o[0] for o in occupations(S)]
    want = T[np.ix_(orb, orb)]
    for H in (S.dense_sc(synth.tbme_table(S.tbme_len, 1)), S.dense_brute(synth.tbme_table(S.tbme_len, 1))):
        np.testing.assert_allclose(H, want, rtol=0, atol=1e-14)
    assert np.abs(want - np.diag(np.diag(want))).max() > 0.1      # off-diagonal (Delta N = 2) couplings present


@pytest.mark.parametrize("Z,N", [(2, 0), (0, 2), (1, 1)])
def test_onebody_two_particle_formula(Z, N):
    """Two particles, no two-body part: <ab|T|cd> = t_ac d_bd - t_ad d_bc -
    t_bc d_ad + t_bd d_ac for a<b, c<d (textbook, with t = 0 across species)."""
    S = oracle.Space(Z, N, 3, 0)
    t1 = synth.onebody_table(S.onebody_len, 8)
    S.set_onebody(t1)
    T = _t_full(S, t1)
    H = S.dense_sc(np.zeros(S.tbme_len, np.float32))
    occ = occupations(S)
    for i, (a, b) in enumerate(occ):
        for j, (c, d) in enumerate(occ):
            want = T[a, c] * (b == d) - T[a, d] * (b == c) - T[b, c] * (a == d) + T[b, d] * (a == c)
            assert H[i, j] == pytest.approx(want, abs=1e-13)


@pytest.mark.parametrize("Z,N,Nmax,twoM", [(2, 2, 2, 0), (3, 3, 2, 0), (2, 1, 3, 1), (3, 2, 2, 3), (1, 2, 3, 7)])
def test_onebody_slater_condon_equals_operator_application(Z, N, Nmax, twoM):
    S = oracle.Space(Z, N, Nmax, twoM)
    S.set_onebody(synth.onebody_table(S.onebody_len, 4))
    t = synth.tbme_table(S.tbme_len, 6)
    Hb = S.dense_brute(t)
    Hs = S.dense_sc(t)
    np.testing.assert_allclose(Hs, Hb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Hb, Hb.T, rtol=0, atol=1e-12)   # Hermiticity
    rp, col, val = S.half_csr(t)                               # the row walk agrees
    Hh = np.zeros_like(Hs)
    for i in range(S.dim):
        Hh[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    np.testing.assert_allclose(np.triu(Hs), Hh, rtol=1e-6, atol=1e-5)


def test_onebody_diagonal_table_equals_orbital_energies():
    """A one-body table with only its diagonal set (t_aa = e_a) gives the
    same matrix as the per-orbital energies."""
    S = oracle.Space(3, 3, 2, 0)
    n = S.norb[0] + S.norb[1]
    esp = synth.single_particle_energies(n, 5)
    t1 = np.zeros(S.onebody_len)
    for a in range(n):
        t1[S.onebody_index(a, a)] = esp[a]
    t = synth.tbme_table(S.tbme_len, 2)
    S.set_onebody(t1)
    H1 = S.dense_sc(t)
    S.set_onebody(None)
    np.testing.assert_array_equal(H1, S.dense_sc(t, esp))
