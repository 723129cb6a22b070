"""Batched persistent solver (scs_batch_*) against the FP64 oracle and the
single-problem solver, through the C ABI.

* FP64 batch with a tight CG follows each program's oracle trajectory to
  1e-9 for 30 iterations (mixed LP / SOC / portfolio programs of uneven
  sizes, all in one launch);
* FP64 batch solves end in the same status and objective as scs_solve;
* FP32 batch of portfolio programs (the uneven-size workload's form): every
  program passes the Sec. 3.5 tests on its original data, objectives match
  the oracle's;
* infeasible and unbounded programs inside a batch return certificates;
* a warm start from the solutions stops at the first test;
* cones other than zero / nonneg / SOC are refused.
"""
import numpy as np
import pytest

from oracle import admm, cones
from paper_1312_3039_gb300 import synth

from test_gpu_parity import TIGHT, check_solution

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scs():
    from paper_1312_3039_gb300 import build, scs as _scs
    build.build()
    return _scs


def mixed_programs():
    rng = np.random.default_rng(3)
    return [synth.lp(0),
            synth.random_cone(11, n=40, cone=synth.Cone(z=5, l=20, q=(3, 7, 1, 2, 40))),
            synth.portfolio(rng, 30),
            synth.portfolio(rng, 57),
            synth.lp(1, n=60, m=90, n_zero=10),
            synth.random_cone(12, n=7, cone=synth.Cone(l=3, q=(4, 2)))]


def as_tuples(progs):
    return [(P.A, P.b, P.c, P.cone) for P in progs]


def test_batch_trajectory_fp64(scs):
    progs = mixed_programs()
    with scs.Batch(as_tuples(progs), **TIGHT) as bt:
        bt.iterate(30)
        got = [bt.iterates(i) for i in range(len(progs))]
    for i, P in enumerate(progs):
        orc = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings())
        for _ in range(30):
            orc.step()
        u, v = got[i]
        eu = np.linalg.norm(u - orc.u) / np.linalg.norm(orc.u)
        ev = np.linalg.norm(v - orc.v) / max(np.linalg.norm(orc.v), 1e-300)
        assert eu <= 1e-9 and ev <= 1e-9, (i, eu, ev)


def test_batch_matches_single_solver_fp64(scs):
    progs = mixed_programs()
    with scs.Batch(as_tuples(progs), precision=0) as bt:
        xs, ys, ss, infos = bt.solve()
    for i, P in enumerate(progs):
        st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=0)
        assert infos[i]["status"] == st == 1, (i, infos[i]["status"], st)
        assert abs(infos[i]["iters"] - info["iters"]) <= 20, (i, infos[i]["iters"], info["iters"])
        assert abs(infos[i]["pobj"] - info["pobj"]) <= 1e-5 * (1 + abs(info["pobj"]))
        check_solution(P, xs[i], ys[i], ss[i])


def test_portfolio_batch_fp32(scs):
    """Every program ends as scs_solve ends it (same status and iteration
    count: the batch runs the same iteration); the solved ones pass the
    Sec. 3.5 tests on their own data and match the oracle's objective.  (A
    few portfolio programs stall near a 1e-3 dual residual and stop at
    max_iters in both solvers.)"""
    progs = synth.portfolio_batch(seed=1, count=96, lo=20, hi=200)
    with scs.Batch(as_tuples(progs), precision=1) as bt:
        xs, ys, ss, infos = bt.solve()
        cfg = bt.config()
    assert cfg["threads"] in (64, 128, 256, 512) and cfg["row_split"] in (4, 16, 64)
    solved = [i for i in range(len(progs)) if infos[i]["status"] == 1]
    assert len(solved) >= 0.9 * len(progs)
    assert all(f["status"] in (1, 2) for f in infos)
    for i in solved:
        check_solution(progs[i], xs[i], ys[i], ss[i], cone_tol=1e-5)
    for i in range(0, len(progs), 8):
        P = progs[i]
        st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=1)
        assert (infos[i]["status"], infos[i]["iters"]) == (st, info["iters"]), (i, infos[i], info)
    for i in solved[::16]:
        ref = admm.solve(progs[i].A, progs[i].b, progs[i].c, progs[i].cone, admm.Settings())
        assert abs(infos[i]["pobj"] - ref.pobj) <= 1e-3 * (1 + abs(ref.pobj)), (i, infos[i]["pobj"], ref.pobj)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_certificates(scs, precision):
    rng = np.random.default_rng(9)
    inf = synth.lp(4, variant="infeasible")
    unb = synth.lp(5, variant="unbounded")
    progs = [synth.lp(6), inf, unb, synth.portfolio(rng, 25)]
    with scs.Batch(as_tuples(progs), precision=precision) as bt:
        xs, ys, ss, infos = bt.solve()
    assert [f["status"] for f in infos] == [1, -1, -2, 1], infos
    y = ys[1]
    assert abs(inf.b @ y + 1.0) < 1e-9
    assert np.linalg.norm(inf.A.T @ y) <= 1e-3
    assert cones.in_Kdual(y, inf.cone, 1e-5 if precision else 1e-6)
    assert np.all(np.isnan(xs[1])) and np.all(np.isnan(ss[1]))
    x = xs[2]
    assert abs(unb.c @ x + 1.0) < 1e-9
    np.testing.assert_allclose(ss[2], -(unb.A @ x), atol=1e-9)
    assert cones.in_K(ss[2], unb.cone, 1e-5)
    assert np.all(np.isnan(ys[2]))


def test_batch_warm_start(scs):
    progs = synth.portfolio_batch(seed=2, count=24, lo=20, hi=120)
    with scs.Batch(as_tuples(progs), precision=1) as bt:
        xs, ys, ss, infos = bt.solve()
        bt.warm_start(xs, ys, ss)
        xs2, ys2, ss2, infos2 = bt.solve()
        # a later cold solve gives the first answer again
        xs3, _, _, infos3 = bt.solve()
    solved = [i for i in range(len(progs)) if infos[i]["status"] == 1]
    assert len(solved) >= 0.8 * len(progs)
    for i in solved:       # restarted from its solution, a program stops at the first test
        assert infos2[i]["status"] == 1 and infos2[i]["iters"] <= 20, (i, infos2[i])
    for i in range(len(progs)):
        assert infos3[i]["iters"] == infos[i]["iters"]
        if i in solved:
            np.testing.assert_array_equal(xs3[i], xs[i])


def test_batch_rejects_other_cones(scs):
    P = synth.random_cone(13, n=10, cone=synth.Cone(l=4, ep=2))
    with pytest.raises(scs.ScsError) as ei:
        scs.Batch(as_tuples([synth.lp(0), P]))
    assert ei.value.code == scs.UNSUPPORTED
