"""ctypes binding of libcih (include/cih.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; torch only
provides device memory and the current stream.  Importing this module loads
``_build/libcih.so`` and raises if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcih.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcih.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python -m paper_1412_5989_gb300.build")

lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_dp = C.POINTER(C.c_double)


class Space(C.Structure):
    _fields_ = [("Z", C.c_int32), ("N", C.c_int32), ("Nmax", C.c_int32), ("twoM", C.c_int32)]


class Instance(C.Structure):
    _fields_ = [("basis", _P), ("K", C.c_int32), ("tbme_dev", _P), ("e_sp_dev", _P), ("evals_host", _dp),
                ("grad_dev", _P), ("nnz", C.c_int64), ("bytes", C.c_int64), ("wave", C.c_int32),
                ("status", C.c_int32)]


_SIGS = {
    "cih_basis_enumerate": [C.POINTER(Space), C.POINTER(_P), _P],
    "cih_basis_host_only": [C.POINTER(Space), C.POINTER(_P)],
    "cih_basis_info": [_P, _i64p, _i32p, _i32p, _i64p, _i64p],
    "cih_basis_tables": [_P, _i32p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), _i32p, _i32p, _i64p],
    "cih_tbme_index": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _i64p, _i32p],
    "cih_basis_destroy": [_P],
    "cih_ham_count": [_P, _P, _i64p, _P],
    "cih_ham_fill": [_P, _P, C.c_int32, C.c_double, _P, _P, _P, _P, _P],
    "cih_ham_fill_interleaved": [_P, _P, C.c_int32, C.c_double, _P, _P, _P, _P, _P],
    "cih_ham_fill_rows": [_P, _P, C.c_int64, C.c_int64, C.c_int32, C.c_double, _P, _P, _P, _P, _P],
    "cih_shard_rows": [_i64p, C.c_int64, C.c_int32, _i64p],
    "cih_onebody_info": [_P, _i64p],
    "cih_onebody_index": [_P, C.c_int32, C.c_int32, _i64p],
    "cih_ham_fill_onebody": [_P, _P, C.c_int32, _P, _P, _P, _P, _P],
    "cih_ham_fill_batched": [_P, _P, C.c_int32, C.c_double, _P, _P, _P, _P, _P],
    "cih_tbme_interleave": [C.c_int32, C.c_int64, _P, _P, _P],
    "cih_ham_build_host": [_P, C.c_int32, C.c_double, _P, _P, _P, _P, _P, C.c_int64, _i64p, _P],
    "cih_set_launch": [_P, C.c_int32, C.c_int32],
    "cih_set_count_mode": [_P, C.c_int32],
    "cih_autotune_fill": [_P, _P, C.c_int32, C.c_double, _P, C.c_int32, _P, _P, _P, _P,
                          _i32p, _i32p, C.POINTER(C.c_float)],
    "cih_check": [_P, _P],
    "cih_batch_solve": [C.POINTER(Instance), C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_double, C.c_int64, _P],
    "cih_lanczos_lowest": [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_double, _dp, _P, _P],
    "cih_lanczos_lowest_em": [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_double, _dp, _P, _P],
    "cih_ham_spmv": [_P, _P, _P, _P, C.c_int32, C.c_int32, _P, _P, _P],
    "cih_ham_upper_sumsq": [_P, _P, C.c_int64, C.c_int64, _P, C.c_int32, C.c_int32, _dp, _P],
    "cih_lanczos_lowest_shard": [_P, _P, C.c_int64, C.c_int64, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                 C.c_double, C.c_double, _P, _P, C.CFUNCTYPE(C.c_int, C.c_void_p), _P, _dp, _P, _P],
    "cih_ham_tbme_grad": [_P, _P, C.c_int32, _P, _P, _P],
    "cih_tridiag_eigen": [C.c_int32, _dp, _dp, _dp, _dp],
    "cih_kernel_launches": [_i64p],
    "cih_rowptr_scan_static": [_P, C.c_int64, _P, _P],
    "cih_strerror": [C.c_int],
    "cih_last_error_detail": [],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_char_p if _name in ("cih_strerror", "cih_last_error_detail") else C.c_int

EXPORTED = sorted(_SIGS)


class CihError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib.cih_strerror(code).decode()
        detail = lib.cih_last_error_detail().decode()
        super().__init__(f"{where}: {msg} ({code}): {detail}")


def _ok(rc: int, where: str) -> int:
    if rc < 0:
        raise CihError(rc, where)
    return rc


def _ptr(t) -> int | None:
    """Device (or host) address of a tensor / array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    return t.ctypes.data


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def kernel_launches() -> int:
    """Kernels libcih has launched in this process so far."""
    n = C.c_int64()
    _ok(lib.cih_kernel_launches(C.byref(n)), "kernel_launches")
    return n.value


def rowptr_scan_static(counts, rowptr=None, stream=None):
    """Row pointers from per-row counts with the scan that allocates no device
    memory (cih_rowptr_scan_static).  counts: int64 CUDA tensor (n,); returns
    (or fills) an int64 CUDA tensor (n + 1,)."""
    import torch
    n = counts.numel()
    if counts.dtype != torch.int64 or not counts.is_cuda or not counts.is_contiguous():
        raise ValueError("counts must be a contiguous int64 CUDA tensor")
    if rowptr is None:
        rowptr = torch.empty(n + 1, dtype=torch.int64, device=counts.device)
    elif (rowptr.dtype != torch.int64 or not rowptr.is_cuda or not rowptr.is_contiguous()
          or rowptr.numel() < n + 1 or rowptr.device != counts.device):
        raise ValueError("rowptr must be a contiguous int64 CUDA tensor of at least n + 1 entries "
                         "on the device of counts")
    with torch.cuda.device(counts.device):
        _ok(lib.cih_rowptr_scan_static(_ptr(counts), n, _ptr(rowptr), _stream(stream)), "rowptr_scan_static")
    return rowptr


def shard_bounds(rowptr_host, nshards: int) -> np.ndarray:
    """Row boundaries of nshards shards of about equal stored nonzeros
    (cih_shard_rows): rowptr_host is a host copy (numpy or CPU tensor) of the
    row pointers; returns int64 (nshards + 1,)."""
    rp = np.ascontiguousarray(np.asarray(rowptr_host), dtype=np.int64)
    out = np.zeros(nshards + 1, dtype=np.int64)
    _ok(lib.cih_shard_rows(rp.ctypes.data_as(_i64p), len(rp) - 1, nshards, out.ctypes.data_as(_i64p)),
        "shard_rows")
    return out


def tbme_interleave(tbme, stream=None):
    """Element-major copy of K tables: out[t * K + k] = tbme[k, t] (device)."""
    import torch
    if tbme.dtype != torch.float32 or not tbme.is_cuda or tbme.dim() != 2 or not tbme.is_contiguous():
        raise ValueError("tbme must be a contiguous float32 CUDA tensor of shape (K, tbme_len)")
    K, n = tbme.shape
    out = torch.empty(max(K * n, 1), dtype=torch.float32, device=tbme.device)
    _ok(lib.cih_tbme_interleave(K, n, _ptr(tbme), _ptr(out), _stream(stream)), "tbme_interleave")
    return out[: K * n]


def tridiag_eigen(diag, offdiag):
    """Eigenvalues (ascending) and eigenvectors (columns) of a symmetric tridiagonal."""
    d = np.ascontiguousarray(diag, dtype=np.float64)
    e = np.ascontiguousarray(offdiag, dtype=np.float64)
    n = len(d)
    w = np.zeros(n)
    Z = np.zeros((n, n))
    _ok(lib.cih_tridiag_eigen(n, d.ctypes.data_as(_dp), e.ctypes.data_as(_dp) if n > 1 else None,
                              w.ctypes.data_as(_dp), Z.ctypes.data_as(_dp)), "tridiag_eigen")
    return w, Z


class Basis:
    """A many-body basis (Z protons, N neutrons, Nmax, 2M) owned by libcih."""

    def __init__(self, Z: int, N: int, Nmax: int, twoM: int, *, host_only: bool = False, stream=None):
        self._h = _P()
        sp = Space(Z, N, Nmax, twoM)
        if host_only:
            _ok(lib.cih_basis_host_only(C.byref(sp), C.byref(self._h)), "basis_host_only")
        else:
            _ok(lib.cih_basis_enumerate(C.byref(sp), C.byref(self._h), _stream(stream)), "basis_enumerate")
        self.Z, self.N, self.Nmax, self.twoM = Z, N, Nmax, twoM
        self.host_only = host_only
        dim = C.c_int64()
        op, on = C.c_int32(), C.c_int32()
        tl = (C.c_int64 * 3)()
        nsd = (C.c_int64 * 2)()
        _ok(lib.cih_basis_info(self._h, C.byref(dim), C.byref(op), C.byref(on), tl, nsd), "basis_info")
        self.dim = dim.value
        self.n_orb = (op.value, on.value)
        self.chan_len = tuple(tl)
        self.tbme_len = sum(self.chan_len)
        self.n_sd = tuple(nsd)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.cih_basis_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host tables ----------------------------------------------------
    def tables(self):
        ntot = self.n_orb[0] + self.n_orb[1]
        orbs = np.zeros((max(ntot, 1), 4), np.int32)
        bp = np.zeros((max(self.n_sd[0], 1), 4), np.uint64)
        bn = np.zeros((max(self.n_sd[1], 1), 4), np.uint64)
        nb = np.zeros(max(self.n_sd[0], 1), np.int32)
        nc = np.zeros(max(self.n_sd[0], 1), np.int32)
        rb = np.zeros(self.n_sd[0] + 1, np.int64)
        _ok(lib.cih_basis_tables(self._h, orbs.ctypes.data_as(_i32p), bp.ctypes.data_as(C.POINTER(C.c_uint64)),
                                 bn.ctypes.data_as(C.POINTER(C.c_uint64)), nb.ctypes.data_as(_i32p),
                                 nc.ctypes.data_as(_i32p), rb.ctypes.data_as(_i64p)), "basis_tables")
        return dict(orbitals=orbs[:ntot], bits_p=bp[: self.n_sd[0]], bits_n=bn[: self.n_sd[1]],
                    nbeg=nb[: self.n_sd[0]], ncnt=nc[: self.n_sd[0]], rowbase=rb)

    @property
    def onebody_len(self) -> int:
        """Entries of the one-body table (cih_onebody_info)."""
        n = C.c_int64()
        _ok(lib.cih_onebody_info(self._h, C.byref(n)), "onebody_info")
        return n.value

    def onebody_index(self, a: int, c: int) -> int:
        """Index of t_ac in the one-body table, -1 if a, c are not one group."""
        idx = C.c_int64()
        _ok(lib.cih_onebody_index(self._h, a, c, C.byref(idx)), "onebody_index")
        return idx.value

    def fill_onebody(self, rowptr, nnz: int, tbme, onebody, stream=None, col=None, val=None):
        """Fill pass with a one-body table (onebody_len float64, CUDA or host)
        in place of the orbital energies (cih_ham_fill_onebody).  Returns
        (col int32[nnz], val float32[K, nnz])."""
        import torch
        t = self._check_table(tbme)
        K = t.shape[0]
        t1 = torch.as_tensor(onebody, dtype=torch.float64).to("cuda").contiguous()
        if t1.numel() != self.onebody_len:
            raise ValueError("the one-body table needs onebody_len entries")
        col, val = self._outputs(nnz, K, col, val)
        _ok(lib.cih_ham_fill_onebody(self._h, _ptr(rowptr), K, _ptr(t), _ptr(t1), _ptr(col), _ptr(val),
                                     _stream(stream)), "ham_fill_onebody")
        return col[:nnz], val[:, :nnz]

    def tbme_index(self, a, b, c, d):
        idx, sg = C.c_int64(), C.c_int32()
        _ok(lib.cih_tbme_index(self._h, a, b, c, d, C.byref(idx), C.byref(sg)), "tbme_index")
        return idx.value, sg.value

    # ---- device passes --------------------------------------------------
    def count(self, stream=None):
        """Count pass + scan: (rowptr int64[dim+1] on the device, nnz)."""
        import torch
        rowptr = torch.empty(self.dim + 1, dtype=torch.int64, device="cuda")
        nnz = C.c_int64()
        _ok(lib.cih_ham_count(self._h, _ptr(rowptr), C.byref(nnz), _stream(stream)), "ham_count")
        return rowptr, nnz.value

    def count_into(self, rowptr, stream=None):
        """Count pass + scan into a caller tensor; no host synchronisation."""
        _ok(lib.cih_ham_count(self._h, _ptr(rowptr), None, _stream(stream)), "ham_count")

    def fill(self, rowptr, nnz: int, tbme, hbar_omega: float = 20.0, e_sp=None, stream=None,
             col=None, val=None):
        """Fill pass.  tbme: (K, tbme_len) or (tbme_len,) float32 CUDA tensor.
        Returns (col int32[nnz], val float32[K, nnz])."""
        import torch
        t = self._check_table(tbme)
        K = t.shape[0]
        col, val = self._outputs(nnz, K, col, val)
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        _ok(lib.cih_ham_fill(self._h, _ptr(rowptr), K, float(hbar_omega), _ptr(t), _ptr(e_sp),
                             _ptr(col), _ptr(val), _stream(stream)), "ham_fill")
        return col[:nnz], val[:, :nnz]

    def fill_rows(self, rowptr, r0: int, r1: int, tbme, hbar_omega: float = 20.0, e_sp=None, stream=None,
                  nnz_s: int | None = None, col=None, val=None):
        """Row-sharded fill (cih_ham_fill_rows): rows r0 .. r1 - 1 only, into
        arrays holding just those rows.  rowptr: the whole row pointers (device);
        nnz_s = rowptr[r1] - rowptr[r0] (read from the device when not given).
        Returns (col int32[nnz_s], val float32[K, nnz_s])."""
        import torch
        t = self._check_table(tbme)
        K = t.shape[0]
        if not (0 <= r0 <= r1 <= self.dim):
            raise ValueError("row range outside 0 .. dim")
        if nnz_s is None:
            nnz_s = int(rowptr[r1].item() - rowptr[r0].item())
        if col is None:
            col = torch.empty(nnz_s, dtype=torch.int32, device="cuda")
        if val is None:
            val = torch.empty((K, nnz_s), dtype=torch.float32, device="cuda")
        if (col.dtype != torch.int32 or val.dtype != torch.float32 or not col.is_cuda or not val.is_cuda
                or col.numel() < nnz_s or val.dim() != 2 or val.shape[0] != K or val.shape[1] != nnz_s
                or not val.is_contiguous()):
            raise ValueError("col must hold nnz_s int32 and val be a contiguous (K, nnz_s) float32 CUDA tensor")
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        if nnz_s > 0:
            _ok(lib.cih_ham_fill_rows(self._h, _ptr(rowptr), r0, r1, K, float(hbar_omega), _ptr(t), _ptr(e_sp),
                                      _ptr(col), _ptr(val), _stream(stream)), "ham_fill_rows")
        return col[:nnz_s], val[:, :nnz_s]

    def _check_table(self, tbme):
        import torch
        t = tbme if tbme.dim() == 2 else tbme.unsqueeze(0)
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[1] != self.tbme_len:
            raise ValueError("tbme must be a contiguous float32 CUDA tensor of shape (K, tbme_len)")
        return t

    def _outputs(self, nnz, K, col, val):
        import torch
        if col is None:
            col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        if val is None:
            val = torch.empty((K, max(nnz, 1)), dtype=torch.float32, device="cuda")
        return col, val

    def fill_interleaved(self, rowptr, nnz: int, tbme_il, K: int, hbar_omega: float = 20.0, e_sp=None,
                         stream=None, col=None, val=None):
        """Fill pass from K element-major tables (tbme_interleave's output,
        float32 (tbme_len * K,)).  Returns (col int32[nnz], val float32[K, nnz])."""
        import torch
        if tbme_il.dtype != torch.float32 or not tbme_il.is_cuda or tbme_il.numel() != K * self.tbme_len:
            raise ValueError("tbme_il must be a float32 CUDA tensor of K * tbme_len entries")
        col, val = self._outputs(nnz, K, col, val)
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        _ok(lib.cih_ham_fill_interleaved(self._h, _ptr(rowptr), K, float(hbar_omega), _ptr(tbme_il.contiguous()),
                                         _ptr(e_sp), _ptr(col), _ptr(val), _stream(stream)), "ham_fill_interleaved")
        return col[:nnz], val[:, :nnz]

    def fill_batched(self, rowptr, nnz: int, tbme_il, K: int, hbar_omega: float = 20.0, e_sp=None,
                     stream=None, col=None, val=None):
        """Batched fill: K element-major tables (tbme_interleave's output) in,
        element-major values out.  Returns (col int32[nnz], val float32[nnz, K])."""
        import torch
        if tbme_il.dtype != torch.float32 or not tbme_il.is_cuda or tbme_il.numel() != K * self.tbme_len:
            raise ValueError("tbme_il must be a float32 CUDA tensor of K * tbme_len entries")
        if col is None:
            col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        if val is None:
            val = torch.empty((max(nnz, 1), K), dtype=torch.float32, device="cuda")
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        _ok(lib.cih_ham_fill_batched(self._h, _ptr(rowptr), K, float(hbar_omega), _ptr(tbme_il.contiguous()),
                                     _ptr(e_sp), _ptr(col), _ptr(val), _stream(stream)), "ham_fill_batched")
        return col[:nnz], val[:nnz]

    def build_to_host(self, tbme, rowptr, col, val, hbar_omega: float = 20.0, e_sp=None, stream=None):
        """End to end with host memory (cih_ham_build_host): tbme (K, tbme_len)
        float32 host array or CPU tensor; rowptr (dim + 1,) int64, col
        (capacity,) int32 and val (K, capacity) float32 host outputs (pinned
        CPU tensors for full speed).  Returns nnz."""
        import torch
        def host(t, dtype):
            if isinstance(t, np.ndarray):
                t = torch.from_numpy(t)
            if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
                raise ValueError("host arrays must be contiguous CPU tensors / arrays of the stated dtype")
            return t
        t = host(tbme, torch.float32)
        t2 = t if t.dim() == 2 else t.unsqueeze(0)
        if t2.shape[1] != self.tbme_len:
            raise ValueError("tbme must have tbme_len entries per set")
        K = t2.shape[0]
        rp, c, v = host(rowptr, torch.int64), host(col, torch.int32), host(val, torch.float32)
        cap = c.numel()
        if rp.numel() != self.dim + 1 or v.numel() != K * cap:
            raise ValueError("rowptr needs dim + 1 entries and val K * capacity")
        es = None if e_sp is None else host(torch.as_tensor(e_sp, dtype=torch.float64), torch.float64)
        nnz = C.c_int64()
        _ok(lib.cih_ham_build_host(self._h, K, float(hbar_omega), _ptr(t2), _ptr(es), _ptr(rp), _ptr(c), _ptr(v),
                                   cap, C.byref(nnz), _stream(stream)), "ham_build_host")
        return nnz.value

    def set_launch(self, warps_per_cta: int, ctas_per_sm: int = 0):
        """Launch shape of this basis' row kernels."""
        _ok(lib.cih_set_launch(self._h, warps_per_cta, ctas_per_sm), "set_launch")

    def set_count_mode(self, walk: bool):
        """Count pass of this basis: walk the candidates (True) or sum the
        count lists where the basis has them (False, the default)."""
        _ok(lib.cih_set_count_mode(self._h, int(bool(walk))), "set_count_mode")

    def autotune_fill(self, rowptr, nnz: int, tbme, hbar_omega: float = 20.0, e_sp=None, *, K: int | None = None,
                      interleaved: bool = False, batched: bool = False, stream=None, col=None, val=None):
        """Time every launch shape of the fill and keep the fastest on this basis.
        tbme: (K, tbme_len) tables, or with interleaved=True the element-major
        copy from tbme_interleave (then K must be given); batched=True times
        the batched fill (interleaved tables, element-major values (nnz, K)).
        Returns (col, val, (warps_per_cta, ctas_per_sm, ms))."""
        import torch
        interleaved = interleaved or batched
        if interleaved:
            if K is None or tbme.numel() != K * self.tbme_len:
                raise ValueError("interleaved tables need K and K * tbme_len entries")
            t = tbme.contiguous()
        else:
            t = self._check_table(tbme)
            K = t.shape[0]
        if batched and val is None:
            val = torch.empty((max(nnz, 1), K), dtype=torch.float32, device="cuda")
        col, val = self._outputs(nnz, K, col, val)
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        w, c, ms = C.c_int32(), C.c_int32(), C.c_float()
        mode = 2 if batched else int(interleaved)
        _ok(lib.cih_autotune_fill(self._h, _ptr(rowptr), K, float(hbar_omega), _ptr(t), mode,
                                  _ptr(e_sp), _ptr(col), _ptr(val), _stream(stream), C.byref(w), C.byref(c),
                                  C.byref(ms)), "autotune_fill")
        v = val[:nnz] if batched else val[:, :nnz]
        return col[:nnz], v, (w.value, c.value, ms.value)

    def check(self, stream=None):
        _ok(lib.cih_check(self._h, _stream(stream)), "check")

    def lanczos(self, rowptr, col, val, nev: int = 5, max_iter: int = 300, tol: float = 1e-8,
                want_vectors: bool = True, stream=None, element_major: bool = False):
        """Lowest nev eigenvalues of each of the K matrices; val is (K, nnz)
        set-major, or (nnz, K) element-major with element_major=True (the
        batched fill's output).  Returns (evals (K, nev) float64 numpy,
        evec0 (K, dim) float64 CUDA or None, converged)."""
        import torch
        v = (val if val.dim() == 2 else val.unsqueeze(0)).contiguous()
        K = v.shape[1] if element_major else v.shape[0]
        ev = np.zeros((K, nev))
        vec = torch.empty((K, self.dim), dtype=torch.float64, device="cuda") if want_vectors else None
        fn = lib.cih_lanczos_lowest_em if element_major else lib.cih_lanczos_lowest
        rc = _ok(fn(self._h, _ptr(rowptr), _ptr(col), _ptr(v), K, nev, max_iter, tol,
                    ev.ctypes.data_as(_dp), _ptr(vec), _stream(stream)), "lanczos_lowest")
        return ev, vec, rc == 0

    def spmv(self, rowptr, col, val, x, element_major: bool = False, stream=None):
        """y = H x from the stored upper half (cih_ham_spmv).  val is (K, nnz)
        set-major or (nnz, K) element-major; x is (dim,) for one set or
        (dim, K) element-major, float64 CUDA.  Returns y shaped like x."""
        import torch
        v = (val if val.dim() == 2 else val.unsqueeze(0)).contiguous()
        K = v.shape[1] if element_major else v.shape[0]
        xx = x.to(torch.float64).contiguous()
        if xx.numel() != self.dim * K or not xx.is_cuda:
            raise ValueError(f"x must hold dim x K = {self.dim} x {K} float64 values on the GPU")
        y = torch.empty_like(xx)
        _ok(lib.cih_ham_spmv(self._h, _ptr(rowptr), _ptr(col), _ptr(v), K, 1 if element_major else 0,
                             _ptr(xx), _ptr(y), _stream(stream)), "ham_spmv")
        return y

    def upper_sumsq(self, rowptr, r0: int, r1: int, val, element_major: bool = False, stream=None) -> float:
        """Sum of the squares of the strictly-upper values of rows r0 .. r1 - 1
        (all sets), val as fill_rows returns it (cih_ham_upper_sumsq)."""
        v = (val if val.dim() == 2 else val.unsqueeze(0)).contiguous()
        K = v.shape[1] if element_major else v.shape[0]
        out = C.c_double()
        _ok(lib.cih_ham_upper_sumsq(self._h, _ptr(rowptr), r0, r1, _ptr(v), K, 1 if element_major else 0,
                                    C.byref(out), _stream(stream)), "ham_upper_sumsq")
        return out.value

    def lanczos_shard(self, rowptr, r0: int, r1: int, col, val, f2: float, combine, nev: int = 5,
                      max_iter: int = 300, tol: float = 1e-8, want_vectors: bool = True, element_major: bool = False,
                      stream=None):
        """This process's part of a Lanczos run over row shards
        (cih_lanczos_lowest_shard).  f2: the whole matrix's sum of
        upper_sumsq over the shards; combine(acc, yx) must replace the two
        buffers (dim * K int64 and float64 CUDA tensors) by their sums over all
        processes.  Returns (evals (K, nev), evec0 (K, dim) or None, converged)."""
        import torch
        v = (val if val.dim() == 2 else val.unsqueeze(0)).contiguous()
        K = v.shape[1] if element_major else v.shape[0]
        acc = torch.zeros(self.dim * K, dtype=torch.int64, device="cuda")
        yx = torch.zeros(self.dim * K, dtype=torch.float64, device="cuda")
        err = []

        def cb(_ctx):
            try:
                combine(acc, yx)
                return 0
            except Exception as e:                                # reported after the call returns
                err.append(e)
                return 1

        cfun = lib.cih_lanczos_lowest_shard.argtypes[14](cb)
        ev = np.zeros((K, nev))
        vec = torch.empty((K, self.dim), dtype=torch.float64, device="cuda") if want_vectors else None
        rc = lib.cih_lanczos_lowest_shard(self._h, _ptr(rowptr), r0, r1, _ptr(col), _ptr(v), K,
                                          1 if element_major else 0, nev, max_iter, tol, float(f2), _ptr(acc),
                                          _ptr(yx), cfun, None, ev.ctypes.data_as(_dp), _ptr(vec), _stream(stream))
        if err:
            raise err[0]
        rc = _ok(rc, "lanczos_lowest_shard")
        return ev, vec, rc == 0

    def tbme_grad(self, rowptr, psi, stream=None):
        """d E0 / d table entry for each set: (K, tbme_len) float64 CUDA tensor."""
        import torch
        p = psi if psi.dim() == 2 else psi.unsqueeze(0)
        p = p.to(torch.float64).contiguous()
        K = p.shape[0]
        g = torch.empty((K, max(self.tbme_len, 1)), dtype=torch.float64, device="cuda")
        _ok(lib.cih_ham_tbme_grad(self._h, _ptr(rowptr), K, _ptr(p), _ptr(g), _stream(stream)), "ham_tbme_grad")
        return g[:, : self.tbme_len]


def solve_batch(items, hbar_omega: float = 20.0, nev: int = 5, max_iter: int = 300, tol: float = 1e-8,
                hbm_budget: int = 0, want_grad: bool = True, stream=None):
    """Fused count -> admission -> fill -> Lanczos -> adjoint over instances of
    different sizes (cih_batch_solve).  items: list of (Basis, tbme (K, tbme_len)
    float32 CUDA tensor[, e_sp]).  Returns (rc, list of dicts with evals (K, nev),
    grad (K, tbme_len) float64 CUDA tensor or None, nnz, bytes, wave, status)."""
    import torch
    n = len(items)
    arr = (Instance * max(n, 1))()
    keep = []
    for i, it in enumerate(items):
        B, t = it[0], it[1]
        e_sp = it[2] if len(it) > 2 else None
        t = B._check_table(t)
        K = t.shape[0]
        ev = np.full((K, nev), np.nan)
        g = torch.empty((K, max(B.tbme_len, 1)), dtype=torch.float64, device="cuda") if want_grad else None
        if e_sp is not None:
            e_sp = e_sp.to(device="cuda", dtype=torch.float64).contiguous()
        keep.append((B, t, ev, g, e_sp))
        arr[i] = Instance(B._h, K, _ptr(t), _ptr(e_sp), ev.ctypes.data_as(_dp), _ptr(g), 0, 0, -1, 0)
    rc = _ok(lib.cih_batch_solve(arr, n, float(hbar_omega), nev, max_iter, float(tol), int(hbm_budget),
                                 _stream(stream)), "batch_solve")
    out = []
    for i, (B, t, ev, g, _) in enumerate(keep):
        x = arr[i]
        out.append(dict(evals=ev, grad=None if g is None else g[:, : B.tbme_len], nnz=x.nnz, bytes=x.bytes,
                        wave=x.wave, status=x.status))
    return rc, out


def lowest_eigenvalue(basis: Basis, tbme, hbar_omega: float = 20.0, e_sp=None, max_iter: int = 400,
                      tol: float = 1e-10):
    """E0 of each of the K matrices, differentiable w.r.t. the two-body tables:
    the backward pass is the library's adjoint (cih_ham_tbme_grad) applied to
    the lowest Ritz vectors.  tbme: (K, tbme_len) or (tbme_len,) float32 CUDA."""
    return _LowestEigenvalue.apply(tbme, basis, float(hbar_omega), e_sp, int(max_iter), float(tol))


def _lowest_eigenvalue_function():
    import torch

    class LowestEigenvalue(torch.autograd.Function):
        @staticmethod
        def forward(ctx, tbme, basis, hbar_omega, e_sp, max_iter, tol):
            t = tbme.detach()
            squeeze = t.dim() == 1
            t = (t.unsqueeze(0) if squeeze else t).contiguous()
            rowptr, col, val, nnz = build_hamiltonian(basis, t, hbar_omega, e_sp)
            ev, psi, conv = basis.lanczos(rowptr, col, val, nev=1, max_iter=max_iter, tol=tol)
            if not conv:
                raise CihError(1, "lowest_eigenvalue: Lanczos did not converge")
            del col, val
            ctx.basis, ctx.squeeze = basis, squeeze
            ctx.save_for_backward(rowptr, psi)
            e0 = torch.from_numpy(ev[:, 0].copy()).to(tbme.device)
            return e0[0] if squeeze else e0

        @staticmethod
        def backward(ctx, g_e):
            rowptr, psi = ctx.saved_tensors
            g = ctx.basis.tbme_grad(rowptr, psi)
            g = g * (g_e.reshape(-1, 1) if g_e.dim() else g_e)
            g = g.to(torch.float32)
            return (g[0] if ctx.squeeze else g), None, None, None, None, None

    return LowestEigenvalue


class _Lazy:
    fn = None

    def apply(self, *a):
        if _Lazy.fn is None:
            _Lazy.fn = _lowest_eigenvalue_function()
        return _Lazy.fn.apply(*a)


_LowestEigenvalue = _Lazy()


def lanczos_distributed(basis: Basis, rowptr, r0: int, r1: int, col, val, nev: int = 5, max_iter: int = 300,
                        tol: float = 1e-8, group=None, want_vectors: bool = True, element_major: bool = False):
    """Lanczos over the row shards of a torch.distributed group: this process
    holds rows r0 .. r1 - 1 (fill_rows); the bound and the two buffers of
    every product are summed with all_reduce (on the device with NCCL, else
    through host copies).  Every process gets the same result."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    f2 = torch.tensor([basis.upper_sumsq(rowptr, r0, r1, val, element_major)], dtype=torch.float64, device=dev)
    dist.all_reduce(f2, group=group)

    def combine(acc, yx):
        if dev == "cuda":
            dist.all_reduce(acc, group=group)
            dist.all_reduce(yx, group=group)
            return
        a, y = acc.cpu(), yx.cpu()
        dist.all_reduce(a, group=group)
        dist.all_reduce(y, group=group)
        acc.copy_(a)
        yx.copy_(y)

    return basis.lanczos_shard(rowptr, r0, r1, col, val, float(f2.item()), combine, nev, max_iter, tol,
                               want_vectors, element_major)


def build_hamiltonian(basis: Basis, tbme, hbar_omega: float = 20.0, e_sp=None, stream=None):
    """Count, scan and fill: (rowptr, col, val, nnz)."""
    rowptr, nnz = basis.count(stream)
    col, val = basis.fill(rowptr, nnz, tbme, hbar_omega, e_sp, stream)
    return rowptr, col, val, nnz
