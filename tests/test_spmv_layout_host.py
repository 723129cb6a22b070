"""The SpMV row layout (built on the host by the same header the kernel uses)
satisfies what the kernel relies on: the stored rows are a permutation of the
matrix rows carrying the same columns; the regions tile the stored rows in
order, every row of a region gets the lane count its length calls for (1 up
to 4 nonzeros, 2 up to 8, tiles of whole rows for 9 to 256, a looping warp up
to 4096, a CTA beyond), every region gets at least one CTA, and the tiles
cover their region in order with whole rows and at most 2048 nonzeros each."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1312_3039_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("hostlayout") / "hostlayout.so"
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                           os.path.join(HERE, "host_layout.cu"), "-o", str(out)])
    return ctypes.CDLL(str(out))


def layout(lib, A, ctas):
    A = sp.csr_matrix(A)
    rows, nnz = A.shape[0], A.nnz
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.indices, dtype=np.int32)
    o_rp = np.zeros(rows + 1, np.int32)
    o_cl = np.zeros(max(nnz, 1), np.int32)
    o_id = np.zeros(max(rows, 1), np.int32)
    info = np.zeros(1 + 4 * 10, np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert lib.host_spmv_layout(rows, P(rp), P(cl), ctas, P(o_rp), P(o_cl), P(o_id), P(info)) == 0
    n = int(info[0])
    regs = [tuple(int(v) for v in info[1 + 4 * k:5 + 4 * k]) for k in range(n)]
    tiles = np.zeros(rows + 2, np.int32)
    nt = lib.host_spmv_tiles(rows, P(rp), P(cl), ctas, P(tiles), rows + 2)
    assert nt >= 0
    return dict(rp=o_rp, cl=o_cl, rowid=o_id[:rows], regs=regs, tiles=tiles[:nt])


TILE = 64           # region tag of the tiles


def lanes_for(n):
    return (1 if n <= 4 else 2 if n <= 8 else TILE if n <= 256 else 33 if n <= 4096 else 256)


def check(A, L):
    A = sp.csr_matrix(A)
    rows = A.shape[0]
    lens = np.diff(A.indptr)
    rid = L["rowid"]
    assert sorted(rid.tolist()) == list(range(rows))
    slen = np.diff(L["rp"])
    np.testing.assert_array_equal(slen, lens[rid])
    for i in range(0, rows, max(1, rows // 300)):
        r = rid[i]
        np.testing.assert_array_equal(L["cl"][L["rp"][i]:L["rp"][i + 1]], A.indices[A.indptr[r]:A.indptr[r + 1]])
    pos = 0
    tiled = [(r0, r1, ctas) for r0, r1, lanes, ctas in L["regs"] if lanes == TILE]
    for r0, r1, lanes, ctas in L["regs"]:
        assert r0 == pos and r1 >= r0 and ctas >= 1
        assert all(lanes_for(int(v)) == lanes for v in slen[r0:r1])
        pos = r1
    assert pos == rows
    t = L["tiles"]
    assert len(tiled) <= 1
    if not tiled:
        assert len(t) == 0
        return
    r0, r1, ctas = tiled[0]
    assert t[0] == r0 and t[-1] == r1 and np.all(np.diff(t) >= 1)
    nz = L["rp"][t[1:]] - L["rp"][t[:-1]]
    assert np.all(nz <= 2048)
    # greedy: a tile ends only where its next row would not fit
    nxt = slen[t[1:-1]]
    assert np.all(nz[:-1] + nxt > 2048)
    assert ctas <= len(t) - 1


@pytest.mark.parametrize("case", ["powerlaw", "uniform", "tiny", "dense_rows", "empty_rows"])
def test_layout_invariants(lib, case):
    rng = np.random.default_rng(3)
    if case == "powerlaw":
        A = synth.powerlaw_rows(rng, 20000, 8000, 200000, max_len=6000)
    elif case == "uniform":
        A = synth.uniform_sparse(rng, 5000, 3000, 60000)
    elif case == "tiny":
        A = sp.csr_matrix(np.array([[1.0, 0, 2], [0, 0, 0], [3, 4, 5]]))
    elif case == "dense_rows":
        A = sp.random(50, 9000, density=0.6, random_state=4, format="csr")
    else:
        A = sp.lil_matrix((3000, 100))
        A[5, :] = 1.0
        A[2999, 3] = 2.0
        A = sp.csr_matrix(A)
    for ctas in (1, 7, 1216):
        check(A, layout(lib, A, ctas))


def test_layout_of_transpose_of_mixed(lib):
    P = synth.mixed_small(0, scale=200)
    for M in (P.A, P.A.T):
        check(M, layout(lib, M, 1216))


def test_threaded_copy_is_identical(lib):
    """The copy into stored order split over host threads gives the same
    layout as one thread, and every stored value is the entry of its own
    row and column (values carry their source positions)."""
    rng = np.random.default_rng(5)
    A = sp.csr_matrix(synth.powerlaw_rows(rng, 30000, 9000, 300000, max_len=5000))
    rows, nnz = A.shape[0], A.nnz
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.indices, dtype=np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    outs = []
    for threads in (1, 3, 8):
        o_rp = np.zeros(rows + 1, np.int32)
        o_cl = np.zeros(nnz, np.int32)
        o_id = np.zeros(rows, np.int32)
        o_v = np.zeros(nnz, np.float64)
        info = np.zeros(1 + 4 * 10, np.int32)
        assert lib.host_spmv_layout_t(rows, P(rp), P(cl), 1216, threads, P(o_rp), P(o_cl), P(o_id), P(info),
                                      P(o_v)) == 0
        outs.append((o_rp, o_cl, o_id, o_v, info))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)
    o_rp, o_cl, o_id, o_v, _ = outs[0]
    src = o_v.astype(np.int64)
    np.testing.assert_array_equal(cl[src], o_cl)
    rows_of_src = np.repeat(np.arange(rows), np.diff(A.indptr))
    rows_of_stored = np.repeat(o_id, np.diff(o_rp))
    np.testing.assert_array_equal(rows_of_src[src], rows_of_stored)


def test_plan_only_layout_matches_the_copying_one(lib):
    """The solver plans its layouts without copying (copy = false) and
    gathers the rows on the device: the plan (row order, row starts,
    regions and their CTAs, tiles) is the copying layout's."""
    rng = np.random.default_rng(9)
    P = synth.mixed_small(0, scale=200)
    cases = [sp.csr_matrix(synth.powerlaw_rows(rng, 30000, 9000, 300000, max_len=5000)), sp.csr_matrix(P.A),
             sp.csr_matrix(P.A.T), sp.csr_matrix(np.array([[1.0, 0, 2], [0, 0, 0], [3, 4, 5]]))]
    for A in cases:
        rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
        cl = np.ascontiguousarray(A.indices, dtype=np.int32)
        for ctas in (1, 7, 1216):
            assert lib.host_spmv_plan_matches(A.shape[0], rp.ctypes.data_as(ctypes.c_void_p),
                                              cl.ctypes.data_as(ctypes.c_void_p), ctas) == 1
