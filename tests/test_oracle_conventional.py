"""Pins of the oracle's conventional potential LBE (Sec. 3.3: the scheme of Chai et al.
with the relaxation time following the permittivity, eps = chi c_s^2 (tau_varphi - 1/2)),
the paper's comparison baseline for its improved scheme (Eq. weq53)."""
import math

import numpy as np
import pytest

import analytic as an
from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl


def params(**kw):
    return ehd.Params.from_dict(wl.make_params(**kw))


def test_reduces_to_the_improved_scheme_for_uniform_eps_and_chi_1():
    """Uniform permittivity and chi = 1: tau_varphi = tau_h and the forcing of Eq. weq53
    vanishes, so both schemes make the same sub-iterations to the last bit."""
    rng = np.random.default_rng(3)
    base = dict(nx=6, ny=10, walls_y=1, eps_v=0.7, eps_l=0.7, varphi_bottom=0.3,
                varphi_top=-0.2, poisson_fixed_iter=25)
    P0, P1 = params(**base), params(**base, potential_scheme=1, chi=1.0)
    phi = rng.uniform(0, 1, (10, 6))
    q = rng.normal(0, 1e-3, (10, 6))
    h0 = ehd.h_eq(rng.normal(0, 0.1, (10, 6))) + rng.normal(0, 1e-3, (9, 10, 6))
    ha, *_ = ehd.poisson_solve(P0, h0, phi, q, (0.3, -0.2))
    hb, *_ = ehd.poisson_solve(P1, h0, phi, q, (0.3, -0.2))
    assert np.array_equal(ha, hb)
    ga, gb = ehd.potential_gradient(P0, ha, phi), ehd.potential_gradient(P1, hb, phi)
    assert np.array_equal(ga[0], gb[0]) and np.array_equal(ga[1], gb[1])


@pytest.mark.parametrize("chi", [0.5, 4.0])
def test_linear_potential_exact_for_any_chi(chi):
    """No charge, uniform permittivity, Dirichlet walls: linear potential to rounding."""
    N = 24
    P = params(nx=4, ny=N, walls_y=1, eps_v=0.5, eps_l=0.5, potential_scheme=1, chi=chi)
    z = np.zeros((N, 4))
    h, it, rel, ok = ehd.poisson_solve(P, np.zeros((9, N, 4)), z, z, (1.0, -0.5), tol=1e-14,
                                       max_iter=500000)
    exact = 1.0 - 1.5 * (np.arange(N) + 0.5) / N
    assert ok and np.abs(ehd.varphi_of(h)[:, 0] - exact).max() < 1e-10


def periodic_mode(N, chi, scheme=1):
    """Uniform eps = 1, periodic N x N, q = -lap v for v = cos(kx + 0.3) sin(ky): the
    relative L2 error of the converged potential and of its local gradient."""
    P = params(nx=N, ny=N, walls_y=0, eps_v=1.0, eps_l=1.0, neutralize_charge=1,
               potential_scheme=scheme, chi=chi)
    k = 2 * math.pi / N
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    v = np.cos(k * x + 0.3) * np.sin(k * y)
    q = 2 * k * k * v
    z = np.zeros((N, N))
    h, it, rel, ok = ehd.poisson_solve(P, np.zeros((9, N, N)), z, q, (0.0, 0.0), tol=1e-12,
                                       max_iter=400000)
    assert ok
    num = ehd.varphi_of(h)
    gx, gy = ehd.potential_gradient(P, h, z)
    vx = -k * np.sin(k * x + 0.3) * np.sin(k * y)
    vy = k * np.cos(k * x + 0.3) * np.cos(k * y)
    return an.rel_l2(num - num.mean(), v), an.rel_l2(np.stack([gx, gy]), np.stack([vx, vy]))


@pytest.mark.parametrize("chi", [0.25, 4.0])
def test_chi_scales_out_of_the_solution(chi):
    """The source is q / chi and the diffusivity eps / chi, so the steady potential solves
    div(eps grad v) + q = 0 whatever chi: a smooth periodic mode converges at second order
    (N = 16 -> 32) and its field is within 1 % at N = 32 (a dropped 1/chi would scale the
    potential by chi).  The potential's error constant grows with tau_varphi (0.02 at
    tau = 1.25, 1.7 at tau = 12.5 for N = 32): the non-equilibrium part of the moving
    populations enters varphi of Eq. weq55."""
    e16, g16 = periodic_mode(16, chi)
    e32, g32 = periodic_mode(32, chi)
    assert g32 < 0.01
    assert math.log2(e16 / e32) > 1.8 and math.log2(g16 / g32) > 1.8


def layers(N, ratio, scheme, chi, tol):
    """Planar diffuse layers between electrodes (as in the potential pins of the improved
    scheme: eps_v = 1, eps_l = ratio eps_v, exact steady charge): iterations to the
    tolerance and the relative L2 errors of varphi and of E."""
    width = 4.0 * N / 32
    p = wl.make_params(nx=4, ny=N, walls_y=1, eps_v=1.0, eps_l=ratio, sigma_v=0.01,
                       sigma_l=0.001, width=width, varphi_bottom=1.0, varphi_top=0.0,
                       potential_scheme=scheme, chi=chi)
    P = ehd.Params.from_dict(p)
    yc = (N - 1) / 2

    def phi_y(s):
        return 0.5 + 0.5 * math.tanh(2 * (yc - s) / width)

    def dphi_y(s):
        return -(1.0 / width) * (1 - math.tanh(2 * (yc - s) / width) ** 2)

    v_ex, q_ex, E_ex = an.planar_diffuse(
        N, phi_y, dphi_y, lambda ph: float(ehd.sigma_of(P, ph)),
        lambda ph: float(ehd.eps_of(P, ph)), lambda ph: float(ehd.deps_dphi(P, ph)),
        lambda ph: P.sigma_l - P.sigma_v, 1.0, 0.0)
    phi = np.repeat(np.array([phi_y(j) for j in range(N)])[:, None], 4, axis=1)
    q = np.repeat(q_ex[:, None], 4, axis=1)
    lin = 1.0 - (np.arange(N) + 0.5) / N
    h0 = ehd.h_eq(np.repeat(lin[:, None], 4, axis=1))
    h, it, rel, ok = ehd.poisson_solve(P, h0, phi, q, (1.0, 0.0), tol=tol, max_iter=2000000)
    assert ok
    gx, gy = ehd.potential_gradient(P, h, phi)
    return it, an.rel_l2(ehd.varphi_of(h)[:, 0], v_ex), an.rel_l2(-gy[:, 0], E_ex)


def test_layers_second_order_with_chi_equal_to_the_ratio():
    """eps ratio 10 with chi = 10 (tau_varphi between 0.53 and 3.5): potential and field
    converge to the diffuse-layer solution at second order (N = 32 -> 64)."""
    _, e32, g32 = layers(32, 10.0, 1, 10.0, 1e-12)
    _, e64, g64 = layers(64, 10.0, 1, 10.0, 1e-12)
    assert math.log2(e32 / e64) > 1.8 and math.log2(g32 / g64) > 1.8
    assert e64 < 0.01 and g64 < 0.01


def test_the_papers_motivation_slow_or_inaccurate_at_large_ratio():
    """Sec. 3.3: with a large permittivity ratio the conventional scheme is slow (chi
    chosen to keep tau_varphi near 1/2 in the low-permittivity phase) or its potential is
    far off (chi = 1: tau_varphi of the high-permittivity phase is large).  eps ratio 20,
    N = 64, iterations to a 1e-10 relative change from a linear start."""
    k0, e0, g0 = layers(64, 20.0, 0, 1.0, 1e-10)       # the paper's scheme
    k1, e1, g1 = layers(64, 20.0, 1, 1.0, 1e-10)       # conventional, chi = 1
    k20, e20, g20 = layers(64, 20.0, 1, 20.0, 1e-10)   # conventional, chi = ratio
    assert k20 > 5 * k0                 # slow
    assert k1 > k0 and e1 > 10 * e0     # inaccurate potential
    for g in (g0, g1, g20):             # all converge to the same field
        assert g < 0.005


def test_planted_mistakes_fail_the_pins(monkeypatch):
    """A dropped 1/chi on the source or a relaxation time that ignores the permittivity
    breaks the pins above."""
    real = ehd.poisson_collide_conventional

    def no_chi(P, h, tau_phi, qsrc):
        return real(P, h, tau_phi, qsrc * P.chi)

    monkeypatch.setattr(ehd, "poisson_collide_conventional", no_chi)
    _, g32 = periodic_mode(32, 4.0)
    assert g32 > 0.5
    monkeypatch.setattr(ehd, "poisson_collide_conventional", real)
    monkeypatch.setattr(ehd, "tau_phi_conventional",
                        lambda P, phi: 0.5 + P.eps_v / (P.chi * ehd.CS2) + 0 * phi)
    _, e64, g64 = layers(64, 10.0, 1, 10.0, 1e-12)
    assert g64 > 0.1
