"""The solver's host-side CSC -> CSR build (compiled for the host with the
device engines stubbed out) against scipy's canonical CSR and CSC, on the CPU:
canonical input, unsorted columns with duplicate entries, empty rows and
columns, at sizes built by one thread and by several."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1312_3039_gb300.scs import CSC, ConeC

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hostbuild") / "hostbuild.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           os.path.join(HERE, "host_build.cu"), "-o", str(out)])
    return C.CDLL(str(out))


def build(lib, m, n, colptr, rowidx, val):
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowidx = np.ascontiguousarray(rowidx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    csc = CSC(m, n, colptr.ctypes.data_as(C.POINTER(C.c_int64)), rowidx.ctypes.data_as(C.POINTER(C.c_int32)),
              val.ctypes.data_as(C.POINTER(C.c_double)))
    zero = np.zeros(1, np.int32)
    zp = np.zeros(1)
    kc = ConeC(m, 0, zero.ctypes.data_as(C.POINTER(C.c_int32)), 0, zero.ctypes.data_as(C.POINTER(C.c_int32)), 0,
               0, 0, zp.ctypes.data_as(C.POINTER(C.c_double)), 0)
    b, c = np.zeros(m), np.zeros(n)
    sizes = np.zeros(3, np.int64)
    rc = lib.host_build(C.byref(csc), b.ctypes.data_as(C.c_void_p), c.ctypes.data_as(C.c_void_p), C.byref(kc),
                        sizes.ctypes.data_as(C.c_void_p))
    if rc != 0:
        return rc, None
    nnz = int(sizes[2])
    out = dict(a_rowptr=np.zeros(m + 1, np.int32), a_col=np.zeros(nnz, np.int32), a_val=np.zeros(nnz),
               at_rowptr=np.zeros(n + 1, np.int32), at_col=np.zeros(nnz, np.int32), at_val=np.zeros(nnz))
    lib.host_build_copy(*(out[k].ctypes.data_as(C.c_void_p) for k in
                          ("a_rowptr", "a_col", "a_val", "at_rowptr", "at_col", "at_val")))
    return rc, out


def expected(m, n, colptr, rowidx, val):
    """scipy's canonical CSR of A and of A^T (sorted indices, duplicates summed)."""
    A = sp.csc_matrix((val, rowidx, colptr), shape=(m, n)).copy()
    A.sum_duplicates()
    R = A.tocsr()
    R.sort_indices()
    return R, A          # CSR of A; the canonical CSC of A is the CSR of A^T


def check(out, R, Acsc):
    assert np.array_equal(out["a_rowptr"], R.indptr)
    assert np.array_equal(out["a_col"], R.indices)
    assert np.array_equal(out["a_val"], R.data)
    assert np.array_equal(out["at_rowptr"], Acsc.indptr)
    assert np.array_equal(out["at_col"], Acsc.indices)
    assert np.array_equal(out["at_val"], Acsc.data)


def random_csc(rng, m, n, nnz, canonical, empty_cols=0):
    """Raw CSC arrays; non-canonical: columns shuffled, with repeated rows.
    Values are small integers so that sums of duplicates are exact."""
    cols = rng.integers(0, n - empty_cols, size=nnz) if n > empty_cols else np.zeros(0, np.int64)
    rows = rng.integers(0, m, size=nnz)
    if not canonical:
        dup = rng.integers(0, nnz, size=nnz // 5)
        cols = np.concatenate([cols, cols[dup]])
        rows = np.concatenate([rows, rows[dup]])
    vals = rng.integers(-8, 9, size=len(rows)).astype(np.float64)
    vals[vals == 0] = 1.0
    if canonical:
        key = np.unique(cols.astype(np.int64) * m + rows)
        cols, rows = key // m, key % m
        vals = rng.integers(-8, 9, size=len(rows)).astype(np.float64)
        vals[vals == 0] = 1.0
        order = np.lexsort((rows, cols))
    else:
        order = np.argsort(cols, kind="stable")     # rows stay in drawn (unsorted) order
    cols, rows, vals = cols[order], rows[order], vals[order]
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, cols + 1, 1)
    return np.cumsum(colptr), rows, vals


@pytest.mark.parametrize("canonical", [True, False])
@pytest.mark.parametrize("size", ["small", "threaded"])
def test_csr_layouts_match_scipy(lib, canonical, size):
    rng = np.random.default_rng(7 + canonical)
    if size == "small":
        m, n, nnz = 300, 170, 2500
    else:
        m, n, nnz = 60_000, 40_000, 1_400_000      # above 2^20 stored entries: several threads
    colptr, rowidx, val = random_csc(rng, m, n, nnz, canonical, empty_cols=7)
    rc, out = build(lib, m, n, colptr, rowidx, val)
    assert rc == 0
    R, Acsc = expected(m, n, colptr, rowidx, val)
    check(out, R, Acsc)


def test_empty_rows_columns_and_no_entries(lib):
    m, n = 5, 4
    rc, out = build(lib, m, n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert rc == 0
    assert np.array_equal(out["a_rowptr"], np.zeros(m + 1)) and np.array_equal(out["at_rowptr"], np.zeros(n + 1))
    # one column holding every row twice, in reverse order
    colptr = np.array([0, 0, 10, 10, 10])
    rowidx = np.array([4, 3, 2, 1, 0, 4, 3, 2, 1, 0])
    val = np.arange(1.0, 11.0)
    rc, out = build(lib, m, n, colptr, rowidx, val)
    assert rc == 0
    R, Acsc = expected(m, n, colptr, rowidx, val)
    check(out, R, Acsc)
    assert np.array_equal(out["at_val"], [15.0, 13.0, 11.0, 9.0, 7.0])


@pytest.mark.parametrize("case", ["row_high", "row_negative", "nan"])
def test_bad_entries_are_refused(lib, case):
    rng = np.random.default_rng(3)
    m, n = 60_000, 40_000
    colptr, rowidx, val = random_csc(rng, m, n, 1_400_000, True)
    rowidx = rowidx.astype(np.int32)
    k = len(rowidx) * 3 // 4                        # in a later part of the threaded check
    if case == "row_high":
        rowidx[k] = m
    elif case == "row_negative":
        rowidx[k] = -1
    else:
        val[k] = np.nan
    rc, _ = build(lib, m, n, colptr, rowidx, val)
    assert rc == -10      # SCS_INVALID_INPUT
