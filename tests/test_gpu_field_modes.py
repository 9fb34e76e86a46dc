"""The field variants (stencil field on varphi, lagged field in hbar) on the GPU: parity
with the oracle at a fixed number of sub-iterations, in both potential loops, and a batch
slot computing the same bits as a stand-alone simulation."""
import numpy as np
import pytest

from paper_2407_01654_gb300 import workloads as wl
from test_gpu_parity import LOOPS, TOL_FIXED, assert_fields, droplet_box, gpu, run_pair  # noqa: F401

pytestmark = pytest.mark.gpu

MODES = [pytest.param(dict(field_mode=1), id="stencil"),
         pytest.param(dict(lagged_field=1), id="lagged"),
         pytest.param(dict(field_mode=1, lagged_field=1), id="stencil+lagged")]


@pytest.mark.parametrize("loop", LOOPS)
@pytest.mark.parametrize("mode", MODES)
def test_droplet_fixed_k(gpu, loop, mode):
    """Ragged 70 x 45 droplet in a field, 100 steps of 3 sub-iterations: every field within
    1e-5 of the oracle."""
    p, f = droplet_box(70, 45, 11.0, seed=6, poisson_fixed_iter=3, poisson_loop=loop, **mode)
    o, g, fo, fg, so, sg = run_pair(gpu, p, f, 100)
    assert_fields(fo, fg, TOL_FIXED)


@pytest.mark.parametrize("mode", MODES)
def test_sessile_ramp_fixed_k(gpu, mode):
    """Ragged 70 x 45 sessile drop while the wall potential ramps (the stencil's ghost rows
    follow it), 60 steps of 4 sub-iterations: within 1e-5 of the oracle."""
    p, f, _ = wl.sessile_drop(nx=70, ny=45, r=14.0, theta=70.0, ramp_steps=60, start_step=10,
                              poisson_fixed_iter=4, **mode)
    f = wl.perturbed(p, f, seed=7, u_amp=1e-3, q_amp=1e-4)
    o, g, fo, fg, so, sg = run_pair(gpu, p, f, 60)
    assert_fields(fo, fg, TOL_FIXED)


def test_batch_slot_matches_single_simulation(gpu):
    """Both variants on: a batch slot and a stand-alone simulation give identical fields."""
    R, S, Ca = wl.droplet_ratios(8)
    p, f, _ = wl.droplet(N=80, r=12.5, R=R, S=S, Ca=Ca, poisson_fixed_iter=4, field_mode=1,
                         lagged_field=1)
    f = wl.perturbed(p, f, seed=8, u_amp=1e-3, q_amp=1e-4)
    b = gpu.Batch(128 << 20, max_slots=2)
    s = b.admit(p, f, 0)
    b.run(40)
    g = gpu.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    g.step(40)
    got, ref = b.read_fields(s), g.read_fields()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
