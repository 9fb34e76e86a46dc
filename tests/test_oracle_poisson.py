"""Pins of the oracle's potential LBE (Eqs. weq52-weq55, Appendix A) against exact
solutions of the variable-permittivity Poisson equation it solves."""
import math

import numpy as np
import pytest

import analytic as an
from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl


def manufactured_periodic(N, eps_ratio=20.0):
    """Periodic N x N, phi(x, y) = 1/2 + 0.45 sin(kx) sin(ky), eps(phi) Hermite with
    ratio eps_l/eps_v = eps_ratio; exact potential v = cos(kx + 0.7) + 0.5 sin(ky + 0.2) and
    the charge q = -div(eps grad v) computed analytically.  Returns the relative L2 errors
    of varphi and of the local gradient (Eq. eqA.16)."""
    p = wl.make_params(nx=N, ny=N, walls_y=0, eps_v=1.0, eps_l=eps_ratio, neutralize_charge=1)
    P = ehd.Params.from_dict(p)
    k = 2 * math.pi / N
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    phi = 0.5 + 0.45 * np.sin(k * x) * np.sin(k * y)
    phx = 0.45 * k * np.cos(k * x) * np.sin(k * y)
    phy = 0.45 * k * np.sin(k * x) * np.cos(k * y)
    v = np.cos(k * x + 0.7) + 0.5 * np.sin(k * y + 0.2)
    vx = -k * np.sin(k * x + 0.7)
    vy = 0.5 * k * np.cos(k * y + 0.2)
    lap = -k * k * np.cos(k * x + 0.7) - 0.5 * k * k * np.sin(k * y + 0.2)
    q = -(ehd.eps_of(P, phi) * lap + ehd.deps_dphi(P, phi) * (phx * vx + phy * vy))
    h, it, rel, ok = ehd.poisson_solve(P, np.zeros((9, N, N)), phi, q, (0.0, 0.0),
                                       tol=1e-11, max_iter=200000)
    assert ok
    num = ehd.varphi_of(h)
    gx, gy = ehd.grad_varphi_local(P, h, ehd.eps_hat_of(P, phi))
    return an.rel_l2(num - num.mean(), v), an.rel_l2(np.stack([gx, gy]), np.stack([vx, vy]))


def layered_walls(N, W0=4.0, N0=32, eps_ratio=10.0, sigma_ratio=0.1):
    """Walls at y = -1/2, N - 1/2 with potentials 1 and 0; tanh layer of width W0 N/N0 at
    mid-height (phase l below); the charge is the exact steady charge of the diffuse
    layers (quadrature solution, tests/analytic.py).  Returns the relative L2 errors of
    varphi and of E = -grad varphi from Eq. eqA.16."""
    width = W0 * N / N0
    p = wl.make_params(nx=4, ny=N, walls_y=1, eps_v=1.0, eps_l=eps_ratio, sigma_v=0.01,
                       sigma_l=0.01 * sigma_ratio, width=width, varphi_bottom=1.0,
                       varphi_top=0.0)
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
    h, it, rel, ok = ehd.poisson_solve(P, h0, phi, q, (1.0, 0.0), tol=1e-12,
                                       max_iter=500000)
    assert ok
    num = ehd.varphi_of(h)[:, 0]
    gx, gy = ehd.grad_varphi_local(P, h, ehd.eps_hat_of(P, phi))
    return an.rel_l2(num, v_ex), an.rel_l2(-gy[:, 0], E_ex)


def test_uniform_eps_linear_potential_exact():
    """No charge, uniform permittivity, Dirichlet walls: the exact solution is linear and
    the anti-bounce-back LBE reproduces it to rounding."""
    N = 24
    P = ehd.Params.from_dict(wl.make_params(nx=4, ny=N, walls_y=1, eps_v=0.5, eps_l=0.5))
    z = np.zeros((N, 4))
    h, it, rel, ok = ehd.poisson_solve(P, np.zeros((9, N, 4)), z, z, (1.0, -0.5),
                                       tol=1e-14, max_iter=500000)
    exact = 1.0 - 1.5 * (np.arange(N) + 0.5) / N
    assert np.abs(ehd.varphi_of(h)[:, 0] - exact).max() < 1e-10


def test_periodic_variable_eps_second_order():
    """Large permittivity ratio (20), periodic manufactured solution: the improved LBE
    (with the discrete forcing) converges to the exact potential at second order, the
    order the paper reports for its potential (Sec. 6.1, Fig. 2b).  The local gradient
    of Eq. eqA.16 converges too; its error constant grows with the first-moment relaxation
    time tau_h + eps_hat/c_s^2 (about 60 here), so its observed order is still rising
    toward 2 on these grids (the one-dimensional layered pin shows 2.0)."""
    errs = [manufactured_periodic(N) for N in (32, 64, 128)]
    ev = [e[0] for e in errs]
    eg = [e[1] for e in errs]
    assert ev[-1] < 0.06 and eg[-1] < 0.06
    assert math.log2(ev[1] / ev[2]) > 1.8
    o1, o2 = math.log2(eg[0] / eg[1]), math.log2(eg[1] / eg[2])
    assert o2 > 1.3 and o2 > o1


def test_layered_walls_second_order():
    """Planar diffuse layers between Dirichlet walls with the exact steady charge: varphi
    and the local field converge at second order as the grid and the interface width are
    refined together."""
    errs = [layered_walls(N) for N in (32, 64, 128)]
    for j in range(2):
        e = [x[j] for x in errs]
        assert math.log2(e[0] / e[1]) > 1.9 and math.log2(e[1] / e[2]) > 1.9
    assert errs[-1][0] < 0.01 and errs[-1][1] < 1e-3


def test_planted_mistake_dropped_forcing_fails(monkeypatch):
    """Planting a mistake in the oracle (the potential LBE without its discrete forcing
    term) makes the layered pin fail: the pin is sensitive to that term."""
    good = layered_walls(64)[0]

    def no_force(P, h, eps_hat):
        z = np.zeros_like(h[0])
        return z, z

    monkeypatch.setattr(ehd, "grad_varphi_local", no_force)
    bad = layered_walls(64)[0]
    assert bad > 20 * good and bad > 0.1


def test_planted_mistake_wrong_wall_rule_fails(monkeypatch):
    """Planting plain bounce-back instead of anti-bounce-back for h breaks the linear
    potential pin."""
    orig = ehd.stream

    def wrong(P, post, kind, varphi_w=(0.0, 0.0)):
        return orig(P, post, "bb")

    monkeypatch.setattr(ehd, "stream", wrong)
    N = 24
    P = ehd.Params.from_dict(wl.make_params(nx=4, ny=N, walls_y=1, eps_v=0.5, eps_l=0.5))
    z = np.zeros((N, 4))
    h, it, rel, ok = ehd.poisson_solve(P, ehd.h_eq(z + 0.2), z, z, (1.0, -0.5), tol=1e-12,
                                       max_iter=200000)
    exact = 1.0 - 1.5 * (np.arange(N) + 0.5) / N
    assert np.abs(ehd.varphi_of(h)[:, 0] - exact).max() > 0.1


def test_stopping_rule():
    """Algorithm 1's rule: the loop stops at the first sub-iteration whose relative change
    sqrt(sum dvarphi^2 / sum varphi^2) is below the tolerance; fixed_iter runs exactly that
    many sub-iterations; max_iter reports non-convergence; 0/0 counts as converged."""
    N = 16
    P = ehd.Params.from_dict(wl.make_params(nx=4, ny=N, walls_y=1, eps_v=0.5, eps_l=0.5))
    z = np.zeros((N, 4))
    q = np.full((N, 4), 1e-3)
    h0 = np.zeros((9, N, 4))
    h, it, rel, ok = ehd.poisson_solve(P, h0, z, q, (0.1, 0.0), tol=1e-4, max_iter=10000)
    assert ok and rel < 1e-4
    # re-run one fewer sub-iteration: its change must be above the tolerance
    h2, it2, rel2, _ = ehd.poisson_solve(P, h0, z, q, (0.1, 0.0), fixed_iter=it - 1)
    assert it2 == it - 1 and rel2 >= 1e-4
    h3, it3, rel3, ok3 = ehd.poisson_solve(P, h0, z, q, (0.1, 0.0), tol=1e-14, max_iter=7)
    assert it3 == 7 and not ok3
    h4, it4, rel4, ok4 = ehd.poisson_solve(P, h0, z, z, (0.0, 0.0))
    assert ok4 and it4 == 1 and rel4 == 0.0


def potential_mean_drift(neutralize):
    """A Gaussian charge bell (net positive charge) in a periodic 32 x 32 box, solved at
    set-up: the mean of varphi then, its change over 200 further sub-iterations, and the
    potential's size."""
    # without neutralisation the rule is met only slowly, as the mean grows: the set-up
    # solve is capped there
    p, f, _, _ = wl.gaussian_bell(32, neutralize_charge=neutralize,
                                  poisson_max_iter=100000 if neutralize else 400)
    s = ehd.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    m0 = float(ehd.varphi_of(s.h).mean())
    h = ehd.poisson_solve(s.P, s.h, f["phi"], f["q"], (0.0, 0.0), fixed_iter=200)[0]
    return m0, float(ehd.varphi_of(h).mean()) - m0, float(np.abs(ehd.varphi_of(h)).max())


def test_periodic_source_is_neutralised():
    """In a periodic box div(eps grad varphi) = -q has a solution only for a source that
    integrates to zero (the left side does).  With the neutralised source q - mean(q) the
    loop settles on a potential whose mean stays at its start value 0: below 1e-12 of the
    potential's size at set-up and after 200 more sub-iterations (measured 1e-18).  The raw
    source with its net charge (the mistake) pumps the mean up without end: by more than
    1e-4 over those sub-iterations."""
    m0, drift, size = potential_mean_drift(1)
    assert abs(m0) < 1e-12 * size and abs(drift) < 1e-12 * size
    m0, drift, size = potential_mean_drift(0)
    assert abs(drift) > 1e-4
