"""The direct subspace step (settings.linsys = 1: (I + A^T A)^-1 formed once
at scs_init and reused, Sec. 4.1 direct method with the factorization
cached, Sec. 4.2) against the oracle's direct method (a sparse factorisation
of the quasi-definite matrix, also cached):

* FP64: both take exact subspace steps, so the trajectories agree to 1e-9 for
  50 iterations (LP, SOC + exponential, every cone type with PSD and power
  blocks, the 1/500 mixed program), graph and plain launches alike;
* full solves: FP64 stops at the oracle's iteration with the objective
  within 1e-4 relative; FP32 within the two-point weak-duality bound; no CG
  step is taken;
* a warm start from the solution reuses the cached inverse and stops at the
  first test; sizes beyond the dense inverse are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm
from paper_1312_3039_gb300 import synth

from test_gpu_parity import check_solution, rel, two_point_bound

pytestmark = pytest.mark.gpu

DIRECT = dict(linsys=1)


@pytest.fixture(scope="module")
def scs():
    from paper_1312_3039_gb300 import build, scs as _scs
    build.build()
    return _scs


def problems():
    return {
        "lp": synth.lp(0),
        "soc_exp": synth.random_cone(11, n=40, cone=synth.Cone(z=5, l=20, q=(3, 7, 1, 2, 40), ep=8)),
        "every_cone": synth.random_cone(31, n=45, cone=synth.Cone(z=4, l=15, q=(3, 5), s=(3,), ep=4, ed=3,
                                                                 p=(0.3, -0.7, 0.5, -0.2, 0.9))),
        "mixed_500": synth.mixed_small(0, scale=500),
    }


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("name", ["lp", "soc_exp", "every_cone", "mixed_500"])
def test_direct_trajectory_fp64(scs, name, use_graph):
    P = problems()[name]
    orc = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings())
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=0, use_graph=use_graph, **DIRECT) as g:
        for k in range(50):
            g.iterate(1)
            orc.step()
            u, v = g.iterates()
            eu = np.linalg.norm(u - orc.u) / np.linalg.norm(orc.u)
            ev = np.linalg.norm(v - orc.v) / max(np.linalg.norm(orc.v), 1e-300)
            assert eu <= 1e-9 and ev <= 1e-9, (k + 1, eu, ev)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["lp", "soc_exp", "every_cone"])
def test_direct_solve(scs, name, precision):
    P = problems()[name]
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision, **DIRECT)
    assert st == scs.SOLVED, info
    check_solution(P, x, y, s, cone_tol=1e-5 if precision else 1e-7)
    assert info["cg_iters"] == 0
    assert info["matvecs"] == 2 * info["iters"] + (info["iters"] + 19) // 20
    ref = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings())
    if precision == 0:
        assert info["iters"] == ref.iters, (info["iters"], ref.iters)
        assert rel(info["pobj"], ref.pobj) <= 1e-4, (info["pobj"], ref.pobj)
    else:
        bound = two_point_bound(P, x, y, s, ref.x, ref.y, ref.s)
        assert abs(info["pobj"] - ref.pobj) <= 1.01 * bound + 1e-9


def test_direct_warm_start_reuses_the_factorization(scs):
    P = synth.lp(3)
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=0, **DIRECT) as g:
        st, x, y, s, info = g.solve()
        assert st == scs.SOLVED
        g.warm_start(x, y, s)
        st2, *_r, info2 = g.solve()
        assert st2 == scs.SOLVED and info2["iters"] <= 20 < info["iters"]
        assert info2["setup_s"] == info["setup_s"]          # no new factorisation


def test_direct_refuses_sizes_beyond_the_dense_inverse(scs):
    n = 8193
    A = sp.identity(n, format="csc")
    with pytest.raises(scs.ScsError) as ei:
        scs.Solver(A, np.ones(n), np.ones(n), synth.Cone(l=n), **DIRECT)
    assert ei.value.code == scs.UNSUPPORTED
