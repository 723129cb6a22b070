"""The learned warm start gains over the method without it: a network
trained (by the library's BF16 kernels) on 2048 solved members of the lasso
family cuts the iterations of 512 held-out members by more than 15% on
average, every warm-started member still passes the Sec. 3.5 tests, and the
warm-started solutions match the cold ones (the cold solve is the fallback:
the solver's own tests decide)."""
import numpy as np
import pytest

from paper_1312_3039_gb300 import synth

pytestmark = pytest.mark.gpu


def test_learned_warm_start_saves_iterations():
    import torch
    from paper_1312_3039_gb300 import build, scs
    from paper_1312_3039_gb300.warmstart import LearnedWarmStart
    build.build()
    fam = synth.lasso_family(0)
    ws = LearnedWarmStart(fam, scs, torch, batch=1024, seed=0)
    try:
        th_tr = fam.thetas(100, 2048)
        th_te = fam.thetas(200, 512)
        infos, _, states = ws.solve_family(th_tr)
        assert all(f["status"] == 1 for f in infos)
        hist = ws.fit(th_tr, states, epochs=60, lr=1e-3)
        assert hist[-1] < 0.6 * hist[0]
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
    finally:
        ws.close()
