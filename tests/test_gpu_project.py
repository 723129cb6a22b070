"""scs_project (device cone projection of a batch of vectors) against the
FP64 oracle's projections onto K and K*, for every cone type of Sec. 6.1:
zero, nonnegative, second-order, exponential and its dual, power and its
dual (and PSD, in test_gpu_psd)."""
import numpy as np
import pytest

from oracle import cones
from paper_1312_3039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


@pytest.mark.parametrize("dual", [0, 1])
def test_project_matches_oracle(env, dual):
    torch, scs = env
    cone = synth.Cone(z=7, l=300, q=(3, 1, 2, 40, 129, 5), ep=50)
    rng = np.random.default_rng(7 + dual)
    count = 9
    V = rng.standard_normal((count, cone.m)) * rng.uniform(0.1, 5.0, size=(count, 1))
    dv = torch.tensor(V, dtype=torch.float64, device="cuda")
    dout = torch.empty_like(dv)
    d2 = scs.project(cone, dual, dv.data_ptr(), dout.data_ptr(), count)
    got = dout.cpu().numpy()
    ref = np.stack([(cones.proj_Kdual if dual else cones.proj_K)(v, cone) for v in V])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(V).max())
    assert abs(d2 - np.sum((ref - V) ** 2)) <= 1e-9 * max(1.0, np.sum((ref - V) ** 2))


def test_project_in_place_and_empty(env):
    torch, scs = env
    cone = synth.Cone(l=5, q=(3,), ep=1)
    V = np.arange(11.0) - 5.0
    dv = torch.tensor(V, dtype=torch.float64, device="cuda")
    scs.project(cone, 0, dv.data_ptr(), dv.data_ptr(), 1)
    np.testing.assert_allclose(dv.cpu().numpy(), cones.proj_K(V, cone), atol=1e-12)
    assert scs.project(cone, 0, dv.data_ptr(), dv.data_ptr(), 0) == 0.0


@pytest.mark.parametrize("dual", [0, 1])
def test_project_power_and_dual_cones_match_oracle(env, dual):
    torch, scs = env
    rng = np.random.default_rng(70 + dual)
    pw = tuple(float(a) for a in rng.uniform(0.02, 0.98, size=40) * rng.choice([-1.0, 1.0], size=40))
    cone = synth.Cone(z=3, l=20, q=(4, 2), ep=10, ed=12, p=pw)
    count = 7
    V = rng.standard_normal((count, cone.m)) * rng.uniform(0.1, 5.0, size=(count, 1))
    V[:, -30:] *= 10.0 ** rng.uniform(-5, 3, size=(count, 30))     # mixed magnitudes on the power rows
    dv = torch.tensor(V, dtype=torch.float64, device="cuda")
    dout = torch.empty_like(dv)
    d2 = scs.project(cone, dual, dv.data_ptr(), dout.data_ptr(), count)
    got = dout.cpu().numpy()
    ref = np.stack([(cones.proj_Kdual if dual else cones.proj_K)(v, cone) for v in V])
    scale = np.maximum(1.0, np.abs(V).max(axis=1, keepdims=True))
    np.testing.assert_allclose(got / scale, ref / scale, rtol=0, atol=1e-11)
    assert abs(d2 - np.sum((ref - V) ** 2)) <= 1e-9 * max(1.0, np.sum((ref - V) ** 2))


def test_project_rejects_bad_power_parameter(env):
    torch, scs = env
    dv = torch.zeros(3, dtype=torch.float64, device="cuda")
    for a in (0.0, 1.0, -1.5, float("nan")):
        with pytest.raises(scs.ScsError) as ei:
            scs.project(synth.Cone(p=(a,)), 0, dv.data_ptr(), dv.data_ptr(), 1)
        assert ei.value.code == scs.INVALID_INPUT
