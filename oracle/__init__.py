"""CPU oracle for the M-scheme CI Hamiltonian -- TEST INFRASTRUCTURE ONLY.

Plain, slow and obviously correct: the C file ``cih_oracle.c`` states the
definitions of the paper's Sec. 1-2 (the many-body Hamiltonian as a finite
symmetric matrix over a Slater-determinant basis, half stored, Lanczos for the
lowest eigenpairs) and this module exposes them through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library in ``paper_1412_5989_gb300``; neither imports
the other.

Every function here is pinned by ``tests/test_oracle_pins.py`` against closed
forms, brute force and library routines; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cih_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
ORW = 8  # words per sub-determinant bit string in the oracle's layout

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP for independent rows only)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    i64p, dp, fp, ip = (C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                        C.POINTER(C.c_float), C.POINTER(C.c_int))
    lp = C.POINTER(C.c_long)
    lib.or_space_new.restype = P
    lib.or_space_new.argtypes = [C.c_int] * 4
    lib.or_space_free.argtypes = [P]
    lib.or_space_info.argtypes = [P, i64p, ip, lp, i64p, i64p]
    lib.or_orbitals.argtypes = [P, C.c_int, ip]
    lib.or_subdets.argtypes = [P, C.c_int, C.POINTER(C.c_uint64), ip, ip]
    lib.or_partner_ranges.argtypes = [P, lp, lp, i64p]
    lib.or_channel_pairs.restype = C.c_long
    lib.or_channel_pairs.argtypes = [P, C.c_int, ip, ip, ip]
    lib.or_basis_state.argtypes = [P, C.c_longlong, lp, lp]
    lib.or_tbme_index.restype = C.c_longlong
    lib.or_tbme_index.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, ip]
    lib.or_element.restype = C.c_int
    lib.or_element.argtypes = [P, fp, dp, C.c_double, C.c_longlong, C.c_longlong, dp]
    lib.or_dense_brute.argtypes = [P, fp, dp, C.c_double, dp]
    lib.or_dense_sc.argtypes = [P, fp, dp, C.c_double, dp]
    lib.or_density_brute.argtypes = [P, dp, dp]
    lib.or_count_rows.argtypes = [P, C.c_longlong, C.c_longlong, i64p]
    lib.or_fill_rows.argtypes = [P, fp, dp, C.c_double, C.c_longlong, C.c_longlong, i64p, ip, fp]
    lib.or_fill_row_list.argtypes = [P, fp, dp, C.c_double, i64p, C.c_long, i64p, ip, fp]
    lib.or_count_row_list.argtypes = [P, i64p, C.c_long, i64p]
    lib.or_jacobi.argtypes = [C.c_int, dp, dp, dp]
    lib.or_lanczos.argtypes = [C.c_longlong, i64p, ip, fp, C.c_int, C.c_int, C.c_double, dp, dp, dp, ip]
    lib.or_half_spmv.argtypes = [C.c_longlong, i64p, ip, fp, dp, dp]
    lib.or_tridiag_eig.restype = C.c_double
    lib.or_tridiag_eig.argtypes = [C.c_int, dp, dp, C.c_int]
    lib.or_grad_elementwise.argtypes = [P, i64p, ip, dp, dp]
    lib.or_onebody_index.restype = C.c_longlong
    lib.or_onebody_index.argtypes = [P, C.c_int, C.c_int]
    lib.or_onebody_len.restype = C.c_longlong
    lib.or_onebody_len.argtypes = [P]
    lib.or_set_onebody.argtypes = [P, dp]
    _lib = lib
    return lib


def _ptr(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def jacobi(A: np.ndarray, vectors: bool = False):
    """Eigenvalues (ascending) and optionally eigenvectors of a symmetric matrix."""
    lib = _load()
    n = A.shape[0]
    M = np.ascontiguousarray(A, dtype=np.float64).copy()
    w = np.zeros(n)
    V = np.zeros((n, n)) if vectors else None
    lib.or_jacobi(n, _ptr(M, C.c_double), _ptr(w, C.c_double), _ptr(V, C.c_double))
    return (w, V) if vectors else w


def tridiag_eig(alpha: np.ndarray, beta: np.ndarray, r: int) -> float:
    """r-th smallest eigenvalue of the tridiagonal (alpha, beta) by bisection."""
    lib = _load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    return lib.or_tridiag_eig(len(a), _ptr(a, C.c_double), _ptr(b, C.c_double), r)


def lanczos(rowptr, col, val, nev=5, max_iter=300, tol=1e-10, v0=None):
    """FP64 Lanczos with full reorthogonalisation on a half-stored CSR matrix.

    Returns (evals[nev], lowest Ritz vector, iterations, converged)."""
    lib = _load()
    dim = len(rowptr) - 1
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    if v0 is None:
        v0 = np.ones(dim)
    v0 = np.ascontiguousarray(v0, dtype=np.float64)
    ev = np.zeros(nev)
    vec = np.zeros(dim)
    it = C.c_int(0)
    rc = lib.or_lanczos(dim, _ptr(rowptr, C.c_longlong), _ptr(col, C.c_int), _ptr(val, C.c_float),
                        nev, max_iter, tol, _ptr(v0, C.c_double), _ptr(ev, C.c_double),
                        _ptr(vec, C.c_double), C.byref(it))
    if rc < 0:
        raise ValueError("oracle lanczos: bad arguments")
    return ev, vec, it.value, rc == 0


def half_spmv(rowptr, col, val, x):
    """y = H x for a half-stored CSR matrix (upper triangle with diagonal), FP64."""
    lib = _load()
    dim = len(rowptr) - 1
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(dim)
    if lib.or_half_spmv(dim, _ptr(rowptr, C.c_longlong), _ptr(col, C.c_int), _ptr(val, C.c_float),
                        _ptr(x, C.c_double), _ptr(y, C.c_double)) < 0:
        raise ValueError("oracle half_spmv: bad arguments")
    return y


class Space:
    """The oracle's many-body space for (Z protons, N neutrons, Nmax, 2M)."""

    def __init__(self, Z: int, N: int, Nmax: int, twoM: int):
        self._lib = _load()
        self._h = self._lib.or_space_new(Z, N, Nmax, twoM)
        if not self._h:
            raise ValueError(f"oracle: cannot build space Z={Z} N={N} Nmax={Nmax} 2M={twoM}")
        self.Z, self.N, self.Nmax, self.twoM = Z, N, Nmax, twoM
        dim = C.c_longlong()
        norb = (C.c_int * 2)()
        nsd = (C.c_long * 2)()
        ch = (C.c_longlong * 3)()
        tl = C.c_longlong()
        self._lib.or_space_info(self._h, C.byref(dim), norb, nsd, ch, C.byref(tl))
        self.dim = dim.value
        self.norb = (norb[0], norb[1])
        self.nsd = (nsd[0], nsd[1])
        self.chan_len = (ch[0], ch[1], ch[2])
        self.tbme_len = tl.value

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_space_free(self._h)
            self._h = None

    # ---- structure -------------------------------------------------
    def orbitals(self, s: int) -> np.ndarray:
        out = np.zeros((max(self.norb[s], 1), 4), dtype=np.int32)
        self._lib.or_orbitals(self._h, s, _ptr(out, C.c_int))
        return out[: self.norb[s]]

    def subdets(self, s: int):
        n = self.nsd[s]
        w = np.zeros((max(n, 1), ORW), dtype=np.uint64)
        Nn = np.zeros(max(n, 1), dtype=np.int32)
        M = np.zeros(max(n, 1), dtype=np.int32)
        self._lib.or_subdets(self._h, s, _ptr(w, C.c_uint64), _ptr(Nn, C.c_int), _ptr(M, C.c_int))
        return w[:n], Nn[:n], M[:n]

    def partner_ranges(self):
        n = self.nsd[0]
        nb = np.zeros(max(n, 1), dtype=np.int64)
        nc = np.zeros(max(n, 1), dtype=np.int64)
        base = np.zeros(n + 1, dtype=np.int64)
        self._lib.or_partner_ranges(self._h, _ptr(nb, C.c_long), _ptr(nc, C.c_long), _ptr(base, C.c_longlong))
        return nb[:n], nc[:n], base

    def channel_pairs(self, c: int):
        n = self._lib.or_channel_pairs(self._h, c, None, None, None)
        pa = np.zeros(max(n, 1), dtype=np.int32)
        pb = np.zeros(max(n, 1), dtype=np.int32)
        g = np.zeros(max(n, 1), dtype=np.int32)
        self._lib.or_channel_pairs(self._h, c, _ptr(pa, C.c_int), _ptr(pb, C.c_int), _ptr(g, C.c_int))
        return pa[:n], pb[:n], g[:n]

    def basis_state(self, i: int):
        p, n = C.c_long(), C.c_long()
        self._lib.or_basis_state(self._h, i, C.byref(p), C.byref(n))
        return p.value, n.value

    def tbme_index(self, a, b, c, d):
        s = C.c_int()
        idx = self._lib.or_tbme_index(self._h, a, b, c, d, C.byref(s))
        return idx, s.value

    # ---- one-body table ---------------------------------------------
    @property
    def onebody_len(self) -> int:
        """Entries of the one-body table: per species, groups of orbitals with
        equal (2m, N parity), each storing its packed upper triangle."""
        return self._lib.or_onebody_len(self._h)

    def onebody_index(self, a: int, c: int) -> int:
        """Table index of t_ac (either order) for combined orbitals, -1 if
        a and c are not one species with equal 2m and N parity."""
        return self._lib.or_onebody_index(self._h, a, c)

    def set_onebody(self, t1=None):
        """Use the one-body table t1 (onebody_len float64) as the one-body part
        of H, H = sum t_ac a+_a a_c + V, for every later matrix call; None
        returns to e_a = hbar_omega (N_a + 3/2) or the per-orbital table."""
        if t1 is None:
            self._t1 = None
            self._lib.or_set_onebody(self._h, None)
            return
        t1 = np.ascontiguousarray(t1, dtype=np.float64)
        if t1.shape != (self.onebody_len,):
            raise ValueError("one-body table needs onebody_len entries")
        self._t1 = t1                                   # kept alive while in use
        self._lib.or_set_onebody(self._h, _ptr(t1, C.c_double))

    # ---- matrix -----------------------------------------------------
    @staticmethod
    def _esp(esp):
        return None if esp is None else np.ascontiguousarray(esp, dtype=np.float64)

    def element(self, tbme, i, j, esp=None, hw=20.0):
        t = np.ascontiguousarray(tbme, dtype=np.float32)
        e = self._esp(esp)
        out = C.c_double()
        rc = self._lib.or_element(self._h, _ptr(t, C.c_float), _ptr(e, C.c_double), hw, i, j, C.byref(out))
        if rc < 0:
            raise RuntimeError("oracle: element lookup outside the table layout")
        return out.value, rc == 1

    def dense_brute(self, tbme, esp=None, hw=20.0) -> np.ndarray:
        t = np.ascontiguousarray(tbme, dtype=np.float32)
        e = self._esp(esp)
        H = np.zeros((self.dim, self.dim))
        self._lib.or_dense_brute(self._h, _ptr(t, C.c_float), _ptr(e, C.c_double), hw, _ptr(H, C.c_double))
        return H

    def dense_sc(self, tbme, esp=None, hw=20.0) -> np.ndarray:
        t = np.ascontiguousarray(tbme, dtype=np.float32)
        e = self._esp(esp)
        H = np.zeros((self.dim, self.dim))
        if self._lib.or_dense_sc(self._h, _ptr(t, C.c_float), _ptr(e, C.c_double), hw, _ptr(H, C.c_double)):
            raise RuntimeError("oracle: element lookup outside the table layout")
        return H

    def count_rows(self, i0=0, i1=None) -> np.ndarray:
        i1 = self.dim if i1 is None else i1
        cnt = np.zeros(max(i1 - i0, 1), dtype=np.int64)
        if self._lib.or_count_rows(self._h, i0, i1, _ptr(cnt, C.c_longlong)):
            raise RuntimeError("oracle: count failed")
        return cnt[: i1 - i0]

    def half_csr(self, tbme, esp=None, hw=20.0):
        """The whole half-stored matrix: (rowptr int64, col int32, val float32)."""
        cnt = self.count_rows()
        rowptr = np.zeros(self.dim + 1, dtype=np.int64)
        np.cumsum(cnt, out=rowptr[1:])
        nnz = int(rowptr[-1])
        col = np.zeros(max(nnz, 1), dtype=np.int32)
        val = np.zeros(max(nnz, 1), dtype=np.float32)
        t = np.ascontiguousarray(tbme, dtype=np.float32)
        e = self._esp(esp)
        if self._lib.or_fill_rows(self._h, _ptr(t, C.c_float), _ptr(e, C.c_double), hw, 0, self.dim,
                                  _ptr(rowptr, C.c_longlong), _ptr(col, C.c_int), _ptr(val, C.c_float)):
            raise RuntimeError("oracle: fill failed")
        return rowptr, col[:nnz], val[:nnz]

    def rows(self, rows, tbme, esp=None, hw=20.0):
        """Selected rows of the half-stored matrix: (counts, offsets, col, val)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cnt = np.zeros(max(len(rows), 1), dtype=np.int64)
        if self._lib.or_count_row_list(self._h, _ptr(rows, C.c_longlong), len(rows), _ptr(cnt, C.c_longlong)):
            raise RuntimeError("oracle: count failed")
        cnt = cnt[: len(rows)]
        off = np.zeros(len(rows) + 1, dtype=np.int64)
        np.cumsum(cnt, out=off[1:])
        n = int(off[-1])
        col = np.zeros(max(n, 1), dtype=np.int32)
        val = np.zeros(max(n, 1), dtype=np.float32)
        t = np.ascontiguousarray(tbme, dtype=np.float32)
        e = self._esp(esp)
        if self._lib.or_fill_row_list(self._h, _ptr(t, C.c_float), _ptr(e, C.c_double), hw,
                                      _ptr(rows, C.c_longlong), len(rows), _ptr(off, C.c_longlong),
                                      _ptr(col, C.c_int), _ptr(val, C.c_float)):
            raise RuntimeError("oracle: fill failed")
        return cnt, off, col[:n], val[:n]

    # ---- gradient ---------------------------------------------------
    def grad_elementwise(self, rowptr, col, psi) -> np.ndarray:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        g = np.zeros(max(self.tbme_len, 1))
        if self._lib.or_grad_elementwise(self._h, _ptr(rowptr, C.c_longlong), _ptr(col, C.c_int),
                                         _ptr(psi, C.c_double), _ptr(g, C.c_double)):
            raise RuntimeError("oracle: gradient lookup outside the table layout")
        return g[: self.tbme_len]

    def density_brute(self, psi) -> np.ndarray:
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        g = np.zeros(max(self.tbme_len, 1))
        self._lib.or_density_brute(self._h, _ptr(psi, C.c_double), _ptr(g, C.c_double))
        return g[: self.tbme_len]
