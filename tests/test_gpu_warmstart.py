"""The learned warm start gains over the method without it.

A network trained (by the library's BF16 kernels) on 2048 members of the
lasso family, solved by the family solver (dense direct step on the CUDA
cores), predicts a scaled starting point for new members:

* family solver: it cuts the iterations of 512 held-out members by more than
  15% on average, every warm-started member still passes the Sec. 3.5 tests,
  and the warm-started solutions match the cold ones;
* plain solver (scs_solve, indirect CG): the prediction is projected onto
  the cones (scs_project), mapped to the caller's units (scs_family_unscale)
  and passed to scs_warm_start (Sec. 4.2); on held-out members this needs
  fewer iterations and less time (inference, projection and mapping
  included) than the cold scs_solve of the same members, and every returned
  point passes the Sec. 3.5 tests recomputed on the host.
The cold-started solve is the fallback: the solver's own tests decide.
"""
import time

import numpy as np
import pytest

from paper_1312_3039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    import torch
    from paper_1312_3039_gb300 import build, scs
    from paper_1312_3039_gb300.warmstart import LearnedWarmStart
    build.build()
    fam = synth.lasso_family(0)
    ws = LearnedWarmStart(fam, scs, torch, batch=1024, seed=0)
    th_tr = fam.thetas(100, 2048)
    infos, _, states = ws.solve_family(th_tr)
    assert all(f["status"] == 1 for f in infos)
    hist = ws.fit(th_tr, states, epochs=60, lr=1e-3)
    assert hist[-1] < 0.6 * hist[0]
    yield fam, ws, scs, torch
    ws.close()


def test_learned_warm_start_saves_family_iterations(trained):
    fam, ws, scs, torch = trained
    th_te = fam.thetas(200, 512)
    cold, _, cstate = ws.solve_family(th_te)
    warm, _, wstate = ws.solve_family(th_te, warm=ws.predict_warm)
    ci = np.array([f["iters"] for f in cold])
    wi = np.array([f["iters"] for f in warm])
    assert all(f["status"] == 1 for f in warm)
    assert wi.mean() < 0.85 * ci.mean(), (wi.mean(), ci.mean())
    # same solutions (scaled x^, normalised): both are 1e-4-accurate answers
    c, w = cstate.cpu().numpy(), wstate.cpu().numpy()
    n = fam.A.shape[1]
    err = np.linalg.norm(c[:, :n] - w[:, :n], axis=1) / np.maximum(np.linalg.norm(c[:, :n], axis=1), 1e-12)
    assert np.median(err) < 1e-2, np.median(err)


def sec35_ok(P, x, y, s, eps=1e-4, slack=1.0001):
    """Sec. 3.5 tests on the original data (FP32 iterates: 1e-4 slack)."""
    nb, nc = np.linalg.norm(P.b), np.linalg.norm(P.c)
    rp = np.linalg.norm(P.A @ x + s - P.b)
    rd = np.linalg.norm(P.A.T @ y + P.c)
    cx, by = P.c @ x, P.b @ y
    return (rp <= eps * (1 + nb) * slack and rd <= eps * (1 + nc) * slack
            and abs(cx + by) <= eps * (1 + abs(cx) + abs(by)) * slack)


def test_learned_warm_start_speeds_up_the_plain_solver(trained):
    fam, ws, scs, torch = trained
    th = fam.thetas(300, 24)
    B, Cs = ws.bc(th)
    n, m = fam.A.shape[1], fam.A.shape[0]
    probs = [fam.problem(t) for t in th]
    solvers = [scs.Solver(P.A, P.b, P.c, P.cone, precision=1) for P in probs]   # scs_init: not timed
    # the held-out members' scaling (sigma, rho per member) for the mapping to the caller's units
    famobj = scs.Family(fam.A, fam.cone, B, Cs, precision=1)
    try:
        cold_t, cold_it = 0.0, []
        for S, P in zip(solvers, probs):
            t0 = time.perf_counter()
            st, x, y, s, info = S.solve()
            cold_t += time.perf_counter() - t0
            assert st == scs.SOLVED
            cold_it.append(info["iters"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, yh, sh = ws.predict_warm(th)               # network, prediction -> scaled point, projections
        X = torch.empty_like(xh)
        Y = torch.empty_like(yh)
        Sv = torch.empty_like(sh)
        famobj.unscale(xh.data_ptr(), yh.data_ptr(), sh.data_ptr(), X.data_ptr(), Y.data_ptr(), Sv.data_ptr())
        Xh, Yh, Sh = X.cpu().numpy(), Y.cpu().numpy(), Sv.cpu().numpy()
        warm_t = time.perf_counter() - t0
        warm_it = []
        for k, (S, P) in enumerate(zip(solvers, probs)):
            t0 = time.perf_counter()
            S.warm_start(Xh[k], Yh[k], Sh[k])
            st, x, y, s, info = S.solve()
            warm_t += time.perf_counter() - t0
            assert st == scs.SOLVED, (k, info)
            assert sec35_ok(P, x, y, s), k
            warm_it.append(info["iters"])
        cold_it, warm_it = np.array(cold_it), np.array(warm_it)
        assert warm_it.mean() < 0.85 * cold_it.mean(), (warm_it.mean(), cold_it.mean())
        assert warm_t < cold_t, (warm_t, cold_t)
    finally:
        famobj.close()
        for S in solvers:
            S.close()
