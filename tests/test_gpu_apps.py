"""The paper's application workloads (Sec. 6.2 - 6.5) on the GPU against the
FP64 oracle, on small instances of each generator: the FP64 engine follows
the oracle's trajectory for 30 iterations (exact subspace solves), and both
engines reach the Sec. 3.5 tests with the objective parity of the other
full-solve tests (FP64: the oracle's iteration count and objective within
1e-4 relative; FP32: within the two-point weak-duality bound)."""
import pytest

from oracle import admm
from paper_1312_3039_gb300 import synth

from test_gpu_parity import assert_objective_parity, check_solution, same_settings, trajectory_parity

pytestmark = pytest.mark.gpu

APPS = {
    "lasso": lambda: synth.lasso_paper(seed=1, p=60, q=30),
    "portfolio": lambda: synth.portfolio_paper(seed=2, p=80, q=6),
    "rpca": lambda: synth.rpca_paper(seed=3, p=10, r=2),
    "logreg": lambda: synth.logreg_paper(seed=4, p=8, q=120),
}


@pytest.fixture(scope="module")
def scs():
    from paper_1312_3039_gb300 import build, scs as _scs
    build.build()
    return _scs


@pytest.mark.parametrize("name", sorted(APPS))
def test_app_trajectory_fp64(scs, name):
    trajectory_parity(scs, APPS[name](), iters=30)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", sorted(APPS))
def test_app_solve(scs, name, precision):
    P = APPS[name]()
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision, max_iters=50000)
    assert st == scs.SOLVED, info
    check_solution(P, x, y, s, cone_tol=1e-5 if precision else 1e-7)
    ref = admm.solve(P.A, P.b, P.c, P.cone, same_settings(max_iters=50000))
    assert_objective_parity(P, precision, info, x, y, s, ref)
