"""The C-ABI library builds, loads and exports every entry point declared in
include/scs_gpu.h; host-side validation rejects bad input before touching a
GPU.  No compute call is made here (these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scs_gpu.h")


@pytest.fixture(scope="module")
def L():
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return scs.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(scs_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(L, name), name


def test_struct_layouts_match_header(tmp_path):
    from paper_1312_3039_gb300 import scs
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "scs_gpu.h"\nint main(void){printf("%zu %zu %zu %zu\\n",'
                   'sizeof(scs_settings), sizeof(scs_info), sizeof(scs_csc), sizeof(scs_cone));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(t) for t in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(scs.Settings), ctypes.sizeof(scs.Info), ctypes.sizeof(scs.CSC), ctypes.sizeof(scs.ConeC)]
    assert got == want


def test_default_settings(L):
    from paper_1312_3039_gb300 import scs
    s = scs.default_settings()
    assert s.alpha == 1.5 and s.cg_rate == 1.5 and s.check_interval == 20
    assert s.eps_pri == s.eps_dual == s.eps_gap == 1e-4
    assert s.precision == 1 and s.normalize == 1


@pytest.mark.parametrize("case", ["cone_rows", "row_index", "nonfinite", "alpha", "colptr", "psd_cond", "precision",
                                  "block_scale", "check_interval", "soc_size", "cg_tol"])
def test_invalid_input_rejected_on_host(L, case):
    from paper_1312_3039_gb300 import scs, synth
    P = synth.lp(0, n=6, m=10, n_zero=2, density=0.5)
    A, b, c, cone = P.A.copy(), P.b.copy(), P.c.copy(), P.cone
    kw = {}
    if case == "cone_rows":
        cone = synth.Cone(z=2, l=7)
    elif case == "row_index":
        A = sp.csc_matrix(A)
        A.indices[0] = 99
    elif case == "nonfinite":
        b[3] = np.nan
    elif case == "alpha":
        kw["alpha"] = 2.5
    elif case == "colptr":
        A = sp.csc_matrix(A)
        A.indptr[2] = A.indptr[3] + 1
    elif case == "psd_cond":
        kw["psd_fp64_cond"] = 0.5
    elif case == "precision":
        kw["precision"] = 2
    elif case == "block_scale":
        kw["block_scale"] = 3
    elif case == "check_interval":
        kw["check_interval"] = 0
    elif case == "soc_size":
        cone = synth.Cone(z=2, l=8, q=(0,))
    elif case == "cg_tol":
        kw["cg_tol_rel"] = -1.0
    with pytest.raises(scs.ScsError) as ei:
        scs.Solver(A, b, c, cone, **kw)
    assert ei.value.code == scs.INVALID_INPUT


def test_psd_order_beyond_the_kernel_is_unsupported(L):
    """A PSD block of order 1025 (above the kernel's 1024) is refused on the
    host with SCS_UNSUPPORTED, before any device work."""
    from paper_1312_3039_gb300 import scs, synth
    k = 1025
    m = k * (k + 1) // 2
    A = sp.csc_matrix((np.ones(3), (np.array([0, 5, m - 1]), np.array([0, 1, 1]))), shape=(m, 2))
    with pytest.raises(scs.ScsError) as ei:
        scs.Solver(A, np.zeros(m), np.ones(2), synth.Cone(s=(k,)))
    assert ei.value.code == scs.UNSUPPORTED


def test_batch_inputs_refused_on_host(L):
    """scs_batch_init checks every program on the host: a bad program is
    refused with its index in the message; exponential cones are not taken
    by the batched solver (SCS_UNSUPPORTED)."""
    from paper_1312_3039_gb300 import scs, synth
    good = synth.lp(0, n=6, m=10, n_zero=2, density=0.5)
    bad = synth.lp(1, n=6, m=10, n_zero=2, density=0.5)
    A = sp.csc_matrix(bad.A.copy())
    A.indices[0] = 99
    with pytest.raises(scs.ScsError) as ei:
        scs.Batch([(good.A, good.b, good.c, good.cone), (A, bad.b, bad.c, bad.cone)])
    assert ei.value.code == scs.INVALID_INPUT
    assert "program 1" in str(ei.value)
    P = synth.random_cone(3, n=12, cone=synth.Cone(l=6, ep=2))
    with pytest.raises(scs.ScsError) as ei:
        scs.Batch([(P.A, P.b, P.c, P.cone)])
    assert ei.value.code == scs.UNSUPPORTED


def test_batch_refusal_names_the_first_failing_program(L):
    """With enough programs that the host checks them on threads (over 2^20
    stored entries in all), the refusal is still the first failing
    program's, as a program-by-program check would report it."""
    from paper_1312_3039_gb300 import scs, synth
    good = synth.lp(2, n=200, m=400, n_zero=20, density=0.05)
    assert good.A.nnz * 300 > 1 << 20
    row_bad = sp.csc_matrix(good.A.copy())
    row_bad.indices[5] = 10_000
    nan_bad = sp.csc_matrix(good.A.copy())
    nan_bad.data[7] = np.nan
    base = [(good.A, good.b, good.c, good.cone)] * 300
    progs = list(base)
    progs[150] = (row_bad, good.b, good.c, good.cone)
    progs[250] = (nan_bad, good.b, good.c, good.cone)
    with pytest.raises(scs.ScsError) as ei:
        scs.Batch(progs)
    assert ei.value.code == scs.INVALID_INPUT
    assert "program 150:" in str(ei.value) and "row index" in str(ei.value)
    expc = synth.random_cone(3, n=12, cone=synth.Cone(l=6, ep=2))
    progs = list(base)
    progs[50] = (expc.A, expc.b, expc.c, expc.cone)
    progs[100] = (nan_bad, good.b, good.c, good.cone)
    with pytest.raises(scs.ScsError) as ei:
        scs.Batch(progs)
    assert ei.value.code == scs.UNSUPPORTED
    assert "program 50:" in str(ei.value)


def test_family_and_network_inputs_refused_on_host(L):
    """scs_family_init refuses cones other than zero / nonnegative / SOC and
    bad data on the host; scs_mlp_create refuses a batch that is not a
    positive multiple of 128 before allocating anything; the product entry
    point refuses shapes outside its tiling and unaligned operands before
    any launch."""
    import ctypes
    from paper_1312_3039_gb300 import scs, synth
    P = synth.random_cone(3, n=12, cone=synth.Cone(l=6, ep=2))
    with pytest.raises(scs.ScsError) as ei:
        scs.Family(P.A, P.cone, P.b[None, :], P.c[None, :])
    assert ei.value.code == scs.UNSUPPORTED
    Q = synth.lp(0, n=6, m=10, n_zero=2, density=0.5)
    bq = Q.b.copy()
    bq[0] = np.inf
    with pytest.raises(scs.ScsError) as ei:
        scs.Family(Q.A, Q.cone, bq[None, :], Q.c[None, :])
    assert ei.value.code == scs.INVALID_INPUT
    err = ctypes.c_int32(0)
    fake_stream = ctypes.c_void_p(1)          # never used: the sizes are refused first
    assert not L.scs_mlp_create(64, 512, 3, 4406, 100, fake_stream, ctypes.byref(err))
    assert err.value == scs.INVALID_INPUT
    f = L.scs_bf16_gemm_async
    # 16-byte aligned stand-in addresses: nothing is dereferenced before the checks fail
    a = 1 << 20
    assert f(a, 64, a, 64, 100, 64, 64, a, 64, 1, a, None) == scs.INVALID_INPUT      # M % 128
    assert f(a, 64, a, 64, 128, 72, 64, a, 72, 1, a, None) == scs.INVALID_INPUT      # N % 64
    assert f(a, 64, a, 64, 128, 64, 48, a, 64, 1, a, None) == scs.INVALID_INPUT      # K % 64 (tcgen05)
    assert f(a + 8, 64, a, 64, 128, 64, 64, a, 64, 1, a, None) == scs.INVALID_INPUT  # unaligned A
    assert f(a, 60, a, 64, 128, 64, 64, a, 64, 1, a, None) == scs.INVALID_INPUT      # lda % 8
