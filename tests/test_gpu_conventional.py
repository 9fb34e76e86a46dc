"""The conventional potential LBE (Sec. 3.3) on the GPU: parity with the oracle, and the
comparison of sub-iterations and accuracy with the paper's scheme."""
import math

import numpy as np
import pytest

import analytic as an
from oracle import ehd as orc
from paper_2407_01654_gb300 import workloads as wl
from test_gpu_parity import (FIELDS, TOL_FIXED, TOL_RULE, assert_fields, droplet_box,  # noqa: F401
                             gpu, run_pair)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("loop", [1, 2, 3], ids=["stream", "resident", "resident2"])
def test_droplet_fixed_k(gpu, loop):
    """Ragged 70 x 45 droplet in a field, chi = 2, 100 steps of 4 sub-iterations: every
    field within 1e-5 of the oracle, on the streaming loop and on the one- and two-step
    on-chip loops."""
    p, f = droplet_box(70, 45, 11.0, seed=2, poisson_fixed_iter=4, potential_scheme=1, chi=2.0,
                       poisson_loop=loop)
    o, g, fo, fg, so, sg = run_pair(gpu, p, f, 100)
    assert_fields(fo, fg, TOL_FIXED)
    assert g.loop_kind() == loop and sg["status"] == 0


def test_loops_compute_the_same_bits(gpu):
    """The conventional collision in the streaming loop and in the one- and two-step
    on-chip loops is the same arithmetic: at a fixed K of 7 (the two-step loop restores
    its parked state) the states after 12 steps on a ragged lattice are bitwise equal."""
    out = []
    for loop in (1, 2, 3):
        p, f = droplet_box(150, 70, 14.0, seed=12, poisson_fixed_iter=7, potential_scheme=1,
                           chi=3.0, poisson_loop=loop)
        g = gpu.Sim(p)
        g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        g.step(12)
        assert g.loop_kind() == loop
        out.append(g.read_fields())
    for k in FIELDS:
        for o in out[1:]:
            assert np.array_equal(out[0][k], o[k]), k


def test_three_step_loop_refuses_the_conventional_scheme(gpu):
    """The three-step loop implements the paper's scheme only: asking for it with the
    conventional scheme is an invalid argument."""
    p, _ = droplet_box(150, 70, 14.0, seed=12, potential_scheme=1, chi=3.0, poisson_loop=4)
    with pytest.raises(gpu.EhdError) as e:
        gpu.Sim(p)
    assert e.value.code == 1


def test_sessile_rule(gpu):
    """Ragged 70 x 45 sessile drop with a rising ramp, chi = 5, the stopping rule: within
    1e-3 of the oracle after 60 steps."""
    p, f, _ = wl.sessile_drop(nx=70, ny=45, r=14.0, theta=70.0, ramp_steps=60, start_step=10,
                              potential_scheme=1, chi=5.0)
    f = wl.perturbed(p, f, seed=4, u_amp=1e-3, q_amp=1e-4)
    o, g, fo, fg, so, sg = run_pair(gpu, p, f, 60)
    assert_fields(fo, fg, TOL_RULE)


def layers_params(N, ratio, scheme, chi):
    width = 4.0 * N / 32
    return wl.make_params(nx=4, ny=N, walls_y=1, eps_v=1.0, eps_l=ratio, sigma_v=0.01,
                          sigma_l=0.001, width=width, varphi_bottom=1.0, varphi_top=0.0,
                          potential_scheme=scheme, chi=chi, poisson_fixed_iter=1)


def layers_gpu(gpu, N, ratio, scheme, chi, tol):
    """Cold solve on the GPU for the planar diffuse layers (exact steady charge): one
    sub-iteration from the linear start inside set_fields, then the loop to `tol`.
    Returns (sub-iterations, relative L2 errors of varphi and E against the exact
    diffuse-layer solution)."""
    p = layers_params(N, ratio, scheme, chi)
    P = orc.Params.from_dict(p)
    width = p["width"]
    yc = (N - 1) / 2

    def phi_y(s):
        return 0.5 + 0.5 * math.tanh(2 * (yc - s) / width)

    def dphi_y(s):
        return -(1.0 / width) * (1 - math.tanh(2 * (yc - s) / width) ** 2)

    v_ex, q_ex, E_ex = an.planar_diffuse(
        N, phi_y, dphi_y, lambda ph: float(orc.sigma_of(P, ph)),
        lambda ph: float(orc.eps_of(P, ph)), lambda ph: float(orc.deps_dphi(P, ph)),
        lambda ph: P.sigma_l - P.sigma_v, 1.0, 0.0)
    phi = np.repeat(np.array([phi_y(j) for j in range(N)])[:, None], 4, axis=1)
    q = np.repeat(q_ex[:, None], 4, axis=1)
    z = np.zeros_like(phi)
    s = gpu.Sim(p)
    s.set_fields(phi, q, z, z)
    it, rel, code = s.solve_potential(tol=tol, max_iter=3000000)
    assert code == 0
    F = s.read_fields(("varphi", "Ey"))
    s.close()
    return 1 + it, an.rel_l2(F["varphi"][:, 0], v_ex), an.rel_l2(F["Ey"][:, 0], E_ex)


@pytest.mark.parametrize("scheme,chi", [(0, 1.0), (1, 20.0)])
def test_cold_solve_matches_the_oracle(gpu, scheme, chi):
    """eps ratio 20, N = 64, the paper's relative change 1e-5: the GPU (FP32) makes the
    oracle's number of sub-iterations to 3 % and reaches its accuracy to 5 %.  (A much
    tighter tolerance is not resolvable in FP32: the change per sub-iteration then sinks
    into the rounding of varphi.)"""
    import test_oracle_conventional as toc
    ko, eo, go = toc.layers(64, 20.0, scheme, chi, 1e-5)
    kg, eg, gg = layers_gpu(gpu, 64, 20.0, scheme, chi, 1e-5)
    assert abs(kg - ko) <= 0.03 * ko, (kg, ko)
    assert abs(eg - eo) <= 0.05 * eo + 1e-4 and abs(gg - go) <= 0.05 * go + 1e-4


@pytest.mark.parametrize("ratio", [20.0, 81.0])
def test_conventional_is_slow_or_inaccurate(gpu, ratio):
    """The paper's motivation (Sec. 3.3) at N = 128 and its tolerance 1e-5 from a cold
    start: chi = ratio (tau_varphi near 1/2 in the low-permittivity phase) needs > 4x the
    sub-iterations of the paper's scheme and gives a worse field; chi = 1 gives a
    potential > 10x less accurate."""
    k0, e0, g0 = layers_gpu(gpu, 128, ratio, 0, 1.0, 1e-5)
    k1, e1, g1 = layers_gpu(gpu, 128, ratio, 1, 1.0, 1e-5)
    kr, er, gr = layers_gpu(gpu, 128, ratio, 1, ratio, 1e-5)
    assert kr > 4 * k0, (kr, k0)
    assert gr > g0, (gr, g0)
    assert e1 > 10 * e0, (e1, e0)
