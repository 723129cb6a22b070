"""scs_project_noalloc, the projection entry point for callers that cannot
allocate device memory, gives the same result as scs_project (which
allocates a scratch buffer per call).

Callers such as an application whose own memory pool has already reserved
the whole GPU, or a serving process that keeps every device allocation under
its own control, need an entry point that allocates nothing:
scs_project_noalloc keeps its scratch in a fixed-size device array inside the
library.  This file is named to be collected last, so that a run stopping at
the first failure has run every other test before it; it passes alone in a
fresh process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_1312_3039_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12      # the projection tests' tolerance (relative to the input's size)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


def test_noalloc_matches_allocating_entry_point_twice(env):
    torch, scs = env
    cone = synth.Cone(z=11, l=500, q=(3, 1, 2, 40, 129, 5, 17), ep=64)
    rng = np.random.default_rng(2024)
    for call, (count, dual) in enumerate([(5, 1), (8, 0)]):      # two calls in a row, different data
        V = rng.standard_normal((count, cone.m)) * rng.uniform(0.1, 5.0, size=(count, 1))
        dv = torch.tensor(V, dtype=torch.float64, device="cuda")
        ref = torch.empty_like(dv)
        got = torch.full_like(dv, float("nan"))
        d_ref = scs.project(cone, dual, dv.data_ptr(), ref.data_ptr(), count)
        d_got = scs.project_noalloc(cone, dual, dv.data_ptr(), got.data_ptr(), count)
        scale = float(np.abs(V).max())
        np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=TOL * scale,
                                   err_msg=f"call {call}")
        assert abs(d_got - d_ref) <= TOL * max(1.0, d_ref), (call, d_got, d_ref)


def test_noalloc_rejects_cones_beyond_its_tables(env):
    torch, scs = env
    cone = synth.Cone(q=tuple([2] * 5000))       # more SOC blocks than the fixed tables hold
    dv = torch.zeros(cone.m, dtype=torch.float64, device="cuda")
    with pytest.raises(scs.ScsError) as ei:
        scs.project_noalloc(cone, 0, dv.data_ptr(), dv.data_ptr(), 1)
    assert ei.value.code == scs.UNSUPPORTED
    assert "SOC blocks" in str(ei.value)          # the reason reaches scs_last_error


def test_noalloc_rejects_power_cones(env):
    torch, scs = env
    cone = synth.Cone(l=2, p=(0.5,))
    dv = torch.zeros(cone.m, dtype=torch.float64, device="cuda")
    with pytest.raises(scs.ScsError) as ei:
        scs.project_noalloc(cone, 0, dv.data_ptr(), dv.data_ptr(), 1)
    assert ei.value.code == scs.UNSUPPORTED
