"""The row-pointer scan that allocates no device memory (cih_rowptr_scan_static)
must give the same row pointers as the scan inside cih_ham_count.

It is meant for callers that cannot allocate GPU memory (their memory belongs
to another framework's pool, or was reserved up front); its scratch is a fixed
array inside the library.  This file is collected last so that a run stopping
at the first failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cih():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_5989_gb300 import cih as mod
    return mod


@pytest.mark.parametrize("sp", [(3, 3, 2, 0), (4, 4, 4, 0)])
def test_static_scan_matches_count_scan(cih, sp):
    B = cih.Basis(*sp)
    rowptr, nnz = B.count()
    counts = (rowptr[1:] - rowptr[:-1]).contiguous()
    # two calls in a row: the shared scratch keeps the first call's contents
    first = cih.rowptr_scan_static(counts)
    second = cih.rowptr_scan_static(counts)
    torch.cuda.synchronize()
    assert torch.equal(first, rowptr) and torch.equal(second, rowptr)
    assert int(first[-1]) == nnz


def test_static_scan_sizes(cih):
    rng = np.random.default_rng(0)
    for n in (0, 1, 4095, 4096, 4097, 1_000_003):            # empty, ragged tiles, many tiles
        c = torch.from_numpy(rng.integers(0, 1000, size=n).astype(np.int64)).cuda()
        out = cih.rowptr_scan_static(c)
        want = np.zeros(n + 1, np.int64)
        np.cumsum(c.cpu().numpy(), out=want[1:])
        assert np.array_equal(out.cpu().numpy(), want)
    inplace = torch.from_numpy(rng.integers(0, 9, size=5000).astype(np.int64)).cuda()
    buf = torch.empty(5001, dtype=torch.int64, device="cuda")
    buf[:5000] = inplace
    cih.rowptr_scan_static(buf[:5000], rowptr=buf)            # in place
    want = np.zeros(5001, np.int64)
    np.cumsum(inplace.cpu().numpy(), out=want[1:])
    assert np.array_equal(buf.cpu().numpy(), want)


def test_static_scan_rejects_oversize(cih):
    big = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(cih.CihError) as e:       # rejected before any device work
        cih._ok(cih.lib.cih_rowptr_scan_static(cih._ptr(big), 67_108_865, cih._ptr(big), cih._stream(None)), "scan")
    assert e.value.code == -3
