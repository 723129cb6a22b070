"""The SpMV work layout (built on the host by the same header the kernel
uses) satisfies every invariant the TMA-staged kernel relies on: every
nonzero is covered exactly once, a run chunk holds whole same-class rows
within the nonzero and row limits, the pieces of a longer row are consecutive
and end with a last piece, per-CTA chunk ranges are monotone, cover all
chunks and never start inside a row, and every 16-byte-aligned copy range
stays inside the padded arrays and fits a shared-memory stage."""
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


def layout(lib, A, grid):
    A = sp.csr_matrix(A)
    rows, nnz = A.shape[0], A.nnz
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.indices, dtype=np.int32)
    pad = 4
    maxc = rows + nnz // 256 + 8
    o_rp = np.zeros(rows + 1 + pad, np.int32)
    o_cl = np.zeros(nnz + pad, np.int32)
    o_id = np.zeros(rows + pad, np.int32)
    o_ch = np.zeros(4 * maxc, np.int32)
    o_kd = np.zeros(maxc, np.int32)
    o_ct = np.zeros(grid + 1, np.int32)
    cnt = np.zeros(8, np.int32)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.host_spmv_layout(rows, P(rp), P(cl), grid, P(o_rp), P(o_cl), P(o_id), P(o_ch), P(o_kd), P(o_ct),
                              P(cnt), maxc)
    assert rc == 0
    nchunk, _, g, cap, rcap, kpad, colw, roww = (int(v) for v in cnt)
    return dict(rp=o_rp, cl=o_cl, rowid=o_id, chunk=o_ch[:4 * nchunk].reshape(-1, 4), kind=o_kd[:nchunk],
                cta=o_ct[:g + 1], nchunk=nchunk, grid=g, cap=cap, rcap=rcap, pad=kpad, colw=colw, roww=roww)


def cls(n):
    return 0 if n <= 1 else int(np.ceil(np.log2(n)))


def check(A, L):
    A = sp.csr_matrix(A)
    rows, nnz = A.shape[0], A.nnz
    lens = np.diff(A.indptr)
    rid = L["rowid"][:rows]
    assert sorted(rid.tolist()) == list(range(rows))
    srp = L["rp"][:rows + 1]
    slen = np.diff(srp)
    np.testing.assert_array_equal(slen, lens[rid])
    for i in range(0, rows, max(1, rows // 200)):          # stored rows carry the right columns
        r = rid[i]
        np.testing.assert_array_equal(L["cl"][srp[i]:srp[i + 1]], A.indices[A.indptr[r]:A.indptr[r + 1]])
    covered = np.zeros(nnz, int)
    row_seen = np.zeros(rows, int)
    chunk_starts_row = np.zeros(L["nchunk"] + 1, bool)
    chunk_starts_row[L["nchunk"]] = True
    expect_next_piece = None
    for c, ((r0, r1, k0, k1), kind) in enumerate(zip(L["chunk"], L["kind"])):
        assert 0 <= k0 <= k1 <= nnz and k1 - k0 <= L["cap"]
        covered[k0:k1] += 1
        if kind == 0:                       # run of whole rows
            assert expect_next_piece is None
            assert r1 > r0 and r1 - r0 <= L["rcap"]
            assert k0 == srp[r0] and k1 == srp[r1]
            assert len({cls(int(v)) for v in slen[r0:r1]}) == 1
            row_seen[r0:r1] += 1
            chunk_starts_row[c] = True
            pa, pb = r0 & ~3, (r1 + 1 + 3) & ~3
            assert pb <= rows + 1 + L["pad"] and pb - pa <= L["roww"]
            ia, ib = r0 & ~3, (r1 + 3) & ~3
            assert ib <= rows + L["pad"] and ib - ia <= L["roww"]
        else:                               # piece of one longer row
            assert kind in (1, 3) and r1 == r0 + 1 and slen[r0] > L["cap"]
            if expect_next_piece is None:
                assert k0 == srp[r0]
                chunk_starts_row[c] = True
            else:
                assert (r0, k0) == expect_next_piece
            expect_next_piece = None if kind == 3 else (r0, k1)
            if kind == 3:
                assert k1 == srp[r1]
                row_seen[r0] += 1
        # 16-byte aligned copy ranges (int32 / fp32: 4 per block, fp64: 2)
        for per in (4, 2):
            a, b = k0 & ~(per - 1), (k1 + per - 1) & ~(per - 1)
            assert b <= nnz + L["pad"] and b - a <= L["colw"]
    assert expect_next_piece is None
    assert np.all(covered == 1) and np.all(row_seen == 1)
    cta = L["cta"]
    assert cta[0] == 0 and cta[-1] == L["nchunk"] and np.all(np.diff(cta) >= 0)
    assert all(chunk_starts_row[c] for c in cta)


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
        A = sp.random(50, 5000, density=0.6, random_state=4, format="csr")
    else:
        A = sp.lil_matrix((3000, 100))
        A[5, :] = 1.0
        A[2999, 3] = 2.0
        A = sp.csr_matrix(A)
    for grid in (1, 7, 456):
        check(A, layout(lib, A, grid))


def test_layout_of_transpose_of_mixed(lib):
    P = synth.mixed_small(0, scale=200)
    for M in (P.A, P.A.T):
        check(M, layout(lib, M, 456))
