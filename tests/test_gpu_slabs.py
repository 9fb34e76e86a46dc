"""Slab decomposition of one lattice (ehd_slabs_*): the lattice computed by 2, 3 or 5
slabs of rows, each with its own buffers and ghost rows, exchanging what crosses each cut
through the C ABI.  With a fixed sub-iteration count every field equals the single
lattice's bit for bit (walls and periodic, the stencil-field variant whose potential
stencil reads across the cuts, ragged slab heights); a neutralised source and the stopping
rule agree within rounding; one case is compared with the oracle directly."""
import numpy as np
import pytest

from oracle import ehd as orc
from paper_2407_01654_gb300 import workloads as wl
from test_gpu_parity import ALL_FIELDS, GROUPS, TOL_FIXED, TOL_RULE, droplet_box, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


def single(gpu, p, f, steps):
    g = gpu.Sim(dict(p, poisson_loop=1))
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    st = g.step(steps)
    out = g.read_fields()
    g.close()
    return st, out


def slabs(gpu, p, f, steps, n):
    t = gpu.Slabs(p, n)
    assert t.set_fields(f["phi"], f["q"], f["ux"], f["uy"]) in (0, 4)
    st = t.step(steps)
    out = t.read_fields()
    t.close()
    return st, out


def periodic_box(nx, ny, seed, **over):
    p = wl.make_params(nx=nx, ny=ny, walls_y=0, rho_l=2.0, rho_v=1.0, mu_l=0.1, mu_v=0.05,
                       eps_l=8.0, eps_v=1.0, sigma_l=0.02, sigma_v=0.01, alpha=0.05,
                       gamma=0.005, width=4.0, **over)
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    phi = wl.tanh_profile(10.0 - np.sqrt((x - 30.0) ** 2 + (y - 18.0) ** 2), 4.0)
    z = np.zeros((ny, nx))
    return p, wl.perturbed(p, dict(phi=phi, q=z + 2e-4, ux=z, uy=z), seed=seed)


CASES = {
    "walls": lambda: droplet_box(70, 45, 11.0, seed=31, poisson_fixed_iter=3),
    "walls_stencil_field": lambda: droplet_box(70, 45, 11.0, seed=32, poisson_fixed_iter=3,
                                               field_mode=1, lagged_field=1),
    "periodic": lambda: periodic_box(66, 40, seed=33, poisson_fixed_iter=4),
    "sessile_ramp": lambda: (lambda pf: (pf[0], wl.perturbed(pf[0], pf[1], seed=34, u_amp=2e-3,
                                                             q_amp=1e-3)))(
        wl.sessile_drop(nx=70, ny=45, r=14.0, theta=70.0, ramp_steps=60, start_step=10,
                        voltage=0.3, ew=0.4, poisson_fixed_iter=2)[:2]),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n", [2, 3, 5])
def test_slabs_equal_single_lattice_bitwise(gpu, case, n):
    p, f = CASES[case]()
    s1, a = single(gpu, p, f, 30)
    s2, b = slabs(gpu, p, f, 30, n)
    assert s2["status"] == 0 and s2["poisson_iters_total"] == s1["poisson_iters_total"]
    for k in ALL_FIELDS:
        assert np.array_equal(a[k], b[k]), k
    # the FP64 phase-mass sum is formed from FP32 per-thread partials, which the slabs
    # partition differently: equal to FP32 rounding
    assert s2["sum_phi"] == pytest.approx(s1["sum_phi"], rel=1e-6)


def test_slabs_neutralised_source_within_rounding(gpu):
    """A periodic lattice with a net charge: the neutralised source's mean charge is summed
    slab by slab, so the fields agree with the single lattice's within rounding."""
    p, f = periodic_box(66, 40, seed=35, poisson_fixed_iter=4, neutralize_charge=1)
    _, a = single(gpu, p, f, 30)
    _, b = slabs(gpu, p, f, 30, 3)
    for g, ks in GROUPS.items():
        assert rel(np.stack([b[k] for k in ks]), np.stack([a[k] for k in ks])) < 1e-6, g


def test_slabs_stopping_rule(gpu):
    """With the paper's stopping rule the slabs' combined sums decide within rounding of the
    single lattice's: total sub-iterations within 2 %, fields within the rule's bar."""
    p, f = droplet_box(64, 48, 10.0, seed=36)
    s1, a = single(gpu, p, f, 25)
    s2, b = slabs(gpu, p, f, 25, 4)
    assert abs(s2["poisson_iters_total"] - s1["poisson_iters_total"]) <= \
        0.02 * s1["poisson_iters_total"] + 2
    for g, ks in GROUPS.items():
        assert rel(np.stack([b[k] for k in ks]), np.stack([a[k] for k in ks])) < TOL_RULE, g


def test_slabs_match_oracle(gpu):
    """Three slabs against the FP64 oracle directly: 100 steps, fixed sub-iteration count,
    relative L2 <= 1e-5 per field."""
    p, f = droplet_box(70, 45, 11.0, seed=37, poisson_fixed_iter=3)
    o = orc.Sim(p)
    o.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    o.step(100)
    fo = o.fields()
    _, fg = slabs(gpu, p, f, 100, 3)
    for g, ks in GROUPS.items():
        assert rel(np.stack([fg[k] for k in ks]), np.stack([fo[k] for k in ks])) <= TOL_FIXED, g


def test_slabs_exchange_bytes(gpu):
    """Bytes crossing the cuts: 2 directions x 8 populations x nx floats per cut and
    sub-iteration; per step, phi (1), (a, q) (2) and 9 pushed populations, each way."""
    p, f = droplet_box(70, 45, 11.0, seed=38, poisson_fixed_iter=3)
    t = gpu.Slabs(p, 3)
    per_it, per_step = t.exchange_bytes()
    t.close()
    assert per_it == 2 * 2 * 8 * 70 * 4 and per_step == 2 * 2 * 12 * 70 * 4
    q, _ = periodic_box(66, 40, seed=39)
    t = gpu.Slabs(q, 3)
    assert t.exchange_bytes()[0] == 3 * 2 * 8 * 66 * 4   # periodic: the wrap is a cut too
    t.close()
