"""Pins of the oracle's charge (Nernst-Planck), Cahn-Hilliard and hydrodynamic LBEs:
closed-form solutions and the exact discrete budgets each LBE must satisfy."""
import math

import numpy as np
import pytest

import analytic as an
from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl


def _sim(p, f, p0=None):
    s = ehd.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"], p0)
    return s


# ---------------------------------------------------------------------------------------
# Nernst-Planck LBE
# ---------------------------------------------------------------------------------------


def gaussian_error(N):
    # The charge is independent of the potential when sigma and eps are uniform
    # (R = -sigma q / eps), so one potential sub-iteration per step suffices here.
    p, f, n, s0 = wl.gaussian_bell(N, poisson_fixed_iter=1)
    s = _sim(p, f)
    s.step(n)
    qa = an.gaussian_bell(N, n, s0, f["q"].max(), p["alpha"], p["sigma_v"], p["eps_v"])
    return an.rel_l2(s.fields()["q"], qa)


def test_gaussian_bell_second_order():
    """Charge relaxation + diffusion of a Gaussian bell (Sec. 6.2, Eq. weq78 with
    diffusion and the exponent read as a decay): second-order convergence under diffusive
    scaling, the order the paper reports (Fig. 3b)."""
    e = [gaussian_error(N) for N in (32, 64, 128)]
    assert e[-1] < 5e-3
    assert math.log2(e[0] / e[1]) > 1.9 and math.log2(e[1] / e[2]) > 1.9


def advected_bell_rates(u=(0.08, 0.04), alpha=0.02, N=64, t1=100, t2=300):
    """A non-conducting (sigma = 0, so R = 0) Gaussian charge bell in a periodic box of
    fluid moving at the uniform velocity u.  The charge equation (Eq. weq56) then
    reduces to dq/dt + div(q u) = alpha lap(q), whose solution's centre moves at u and
    whose variance grows by 2 alpha per unit time along each axis.  Returns, per axis, the
    centre's speed over u and the variance's growth rate over 2 alpha, both measured from
    step t1 (past the start transient of the initial equilibrium populations) to t2, the
    moments taken about the exact centre with periodic wrapping."""
    p, f, _, _ = wl.gaussian_bell(N, alpha=alpha, sigma_l=0.0, sigma_v=0.0,
                                  poisson_fixed_iter=2)
    z = np.zeros((N, N))
    f = dict(f, ux=z + u[0], uy=z + u[1])
    x, y = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float))
    s = _sim(p, f)

    def moments(t):
        q = s.fields()["q"]
        Q = q.sum()
        out = []
        for coord, ui in ((x, u[0]), (y, u[1])):
            d = (coord - (N / 2 + ui * t) + N / 2) % N - N / 2
            m = (q * d).sum() / Q
            out.append((N / 2 + ui * t + m, (q * (d - m) ** 2).sum() / Q))
        return out

    s.step(t1)
    a = moments(t1)
    s.step(t2 - t1)
    b = moments(t2)
    dt = t2 - t1
    speed = [(b[k][0] - a[k][0]) / dt / u[k] for k in range(2)]
    spread = [(b[k][1] - a[k][1]) / (2 * alpha * dt) for k in range(2)]
    return speed, spread


def test_advected_charge_bell_moves_and_spreads_exactly():
    """Advection-diffusion of a charge bell at a uniform velocity: the centre moves at u
    and the variance grows at 2 alpha per step along each axis, within 1e-5 (measured
    2e-7 and 6e-8).  This pins the velocity term of the charge equilibrium (Eq. weq61)
    and the time derivative of the charge flux in the forcing term T_i (Eq. weq60, a
    backward difference), which cancels the lattice's numerical diffusion."""
    speed, spread = advected_bell_rates()
    assert max(abs(v - 1) for v in speed) < 1e-5, speed
    assert max(abs(v - 1) for v in spread) < 1e-5, spread


def test_planted_mistake_charge_flux_time_difference_fails(monkeypatch):
    """Planted mistake: the time derivative of the charge flux q u left out of T_i
    (Eq. weq60; every step taken as the first, so (qu)^n - (qu)^(n-1) = 0).
    The bell still moves at u, but it spreads too slowly by 3 u_i^2 along axis i
    (1.9 % along x at u_x = 0.08)."""
    orig = ehd.Sim._one_step

    def wrong(self):
        self.history_valid = False
        return orig(self)

    monkeypatch.setattr(ehd.Sim, "_one_step", wrong)
    speed, spread = advected_bell_rates()
    assert abs(spread[0] - 1) > 1e-2


def _charge_budget_case(seed=5):
    p, f, info = wl.droplet(N=24, r=6.0, R=3.0, S=0.5, Ca=0.3)
    p["alpha"] = 0.05
    f = wl.perturbed(p, f, seed=seed, u_amp=3e-3, q_amp=2e-3)
    return p, f


def test_charge_budget_exact():
    """Exact discrete charge budget of the NP LBE (Eqs. weq58-weq62 with the lagged R of
    Algorithm 1): sum_x sum_i l changes per step by sum_x [R^{n-1}/(2 tau_l) +
    (1 - 1/(2 tau_l)) R^n]; streaming with bounce-back conserves the total."""
    p, f = _charge_budget_case()
    s = _sim(p, f)
    for _ in range(4):
        before = s.l.sum()
        R_prev = s.R_prev.copy()
        s.step(1)
        tl = s.P.tau_l
        expected = np.sum(R_prev / (2 * tl) + (1 - 1 / (2 * tl)) * s.R_prev)
        scale = np.abs(s.l).sum()
        assert abs((s.l.sum() - before) - expected) < 1e-12 * scale


def test_planted_mistake_charge_closure_fails(monkeypatch):
    """Dropping the R/2 correction of the charge moment (Eq. weq62) breaks the charge
    budget pin."""
    orig = ehd.Sim._moments

    def wrong(self):
        phi, q, rho, ux, uy = orig(self)
        return phi, q - 0.5 * self.R_prev, rho, ux, uy

    monkeypatch.setattr(ehd.Sim, "_moments", wrong)
    p, f = _charge_budget_case()
    s = _sim(p, f)
    s.step(1)
    worst = 0.0
    for _ in range(3):
        before = s.l.sum()
        R_prev = s.R_prev.copy()
        s.step(1)
        tl = s.P.tau_l
        expected = np.sum(R_prev / (2 * tl) + (1 - 1 / (2 * tl)) * s.R_prev)
        worst = max(worst, abs((s.l.sum() - before) - expected) / np.abs(s.l).sum())
    assert worst > 1e-9


# ---------------------------------------------------------------------------------------
# Cahn-Hilliard LBE
# ---------------------------------------------------------------------------------------


def test_phase_mass_budget_exact():
    """Exact discrete budget of the well-balanced CH LBE (Eq. weq45, sum G_i = -u.grad phi):
    sum_x phi^{n+1} - sum_x phi^n = -sum_x [s^n + (s^n - s^{n-1})/2], s = u.grad phi,
    with s^{-1} = s^0 at the first step.  (Without flow the phase mass is conserved.)"""
    p, f = _charge_budget_case(seed=11)
    s = _sim(p, f)
    scale = np.abs(s.g).sum()
    for k in range(4):
        before = s.g.sum()
        s_prev = s.s_prev.copy()
        first = not s.history_valid
        s.step(1)
        s_now = s.s_prev
        sp = s_now if first else s_prev
        expected = -np.sum(s_now + 0.5 * (s_now - sp))
        assert abs((s.g.sum() - before) - expected) < 1e-12 * scale


def test_phase_mass_conserved_without_flow():
    """No flow, no field: sum phi is conserved to rounding (1e-12 relative)."""
    p, f = wl.planar_layers(nx=6, ny=20, varphi_high=0.0)
    s = _sim(p, f)
    m0 = s.g.sum()
    s.step(50)
    # the flow induced by the diffuse interface is at the rounding level here
    assert abs(s.g.sum() - m0) < 1e-12 * abs(m0)


def test_planted_mistake_ch_source_sign_fails(monkeypatch):
    """Flipping the sign of the CH source G_i breaks the phase-mass budget pin."""
    orig = ehd.g_source
    monkeypatch.setattr(ehd, "g_source", lambda s_adv: -orig(s_adv))
    p, f = _charge_budget_case(seed=11)
    s = _sim(p, f)
    before = s.g.sum()
    s.step(1)
    s_now = s.s_prev
    expected = -np.sum(s_now)
    assert abs((s.g.sum() - before) - expected) > 1e-9 * np.abs(s.g).sum()


def test_flat_interface_stationary():
    """The tanh profile 1/2 + 1/2 tanh(2y/W) is the CH equilibrium of the double-well free
    energy with kappa and beta of Sec. 2.2; the LBE keeps it to O(dx^2/W^2): the drift
    after 500 steps is small and falls by more than 4x when W doubles."""
    drift = []
    for W in (4.0, 8.0):
        p, f = wl.planar_layers(nx=4, ny=64, width=W, varphi_high=0.0)
        s = _sim(p, f)
        s.step(500)
        drift.append(np.abs(s.fields()["phi"] - f["phi"]).max())
    assert drift[0] < 1e-2 and drift[0] / drift[1] > 4.0


def ch_cosine_decay_error(N, amp=1e-3, t1=50, t2=450):
    """A small cosine amp cos(2 pi x / N) on the bulk phase phi = 0 (periodic N x 4, no
    flow to speak of, no charge).  Linearising the CH equation about phi = 0, where the
    bulk free energy's second derivative is 2 beta, the mode decays as exp(-lambda t) with
    lambda = M k^2 (2 beta + kappa k^2) (Sec. 2.2; M the mobility of Sec. 3.2).  Returns
    the relative error of the measured rate from step t1 to t2."""
    ny = 4
    p = wl.make_params(nx=N, ny=ny, walls_y=0, rho_l=1.0, rho_v=1.0, mu_l=0.1, mu_v=0.1,
                       eps_l=1.0, eps_v=1.0, sigma_l=0.0, sigma_v=0.0, alpha=0.02,
                       gamma=0.01, width=4.0, mobility=0.05, poisson_fixed_iter=1,
                       neutralize_charge=1)
    x = np.meshgrid(np.arange(N, dtype=float), np.arange(ny, dtype=float))[0]
    k = 2 * math.pi / N
    z = np.zeros((ny, N))
    s = _sim(p, dict(phi=amp * np.cos(k * x), q=z, ux=z, uy=z))

    def amplitude():
        return 2 * (s.fields()["phi"][0] * np.cos(k * x[0])).mean()

    s.step(t1)
    a1 = amplitude()
    s.step(t2 - t1)
    a2 = amplitude()
    P = s.P
    lam = -math.log(a2 / a1) / (t2 - t1)
    return lam / (P.mobility * k * k * (2 * P.beta + P.kappa * k * k)) - 1


def test_ch_cosine_mode_decays_at_the_linearised_rate():
    """The linearised CH decay rate M k^2 (2 beta + kappa k^2): within 5e-3 at N = 64 and
    1e-3 at N = 128 (measured 1.3e-3 and 3.4e-4: second order).  This pins the CH
    relaxation time against the mobility (M = c_s^2 (tau_g - 1/2)) and the chemical
    potential's bulk and gradient terms together."""
    assert abs(ch_cosine_decay_error(64)) < 5e-3
    assert abs(ch_cosine_decay_error(128)) < 1e-3


def translated_band_spread_change(u0=0.05, N=64, t1=100, t2=300):
    """A band of phase l (20 nodes wide, two flat interfaces of width 4, uniform density
    and viscosity, no charge) in a periodic N x 4 box of fluid moving at u0 along x.  The
    coupled equations translate it unchanged (uniform flow carries the equilibrium
    profile along).  Returns the change of the profile's variance about its centre (a
    measure of its width, about 33 here) from step t1 to step t2, the moments taken about
    the translated centre with periodic wrapping."""
    ny = 4
    p = wl.make_params(nx=N, ny=ny, walls_y=0, rho_l=1.0, rho_v=1.0, mu_l=0.1, mu_v=0.1,
                       eps_l=1.0, eps_v=1.0, sigma_l=0.0, sigma_v=0.0, alpha=0.02,
                       gamma=0.01, width=4.0, mobility=0.05, poisson_fixed_iter=1,
                       neutralize_charge=1)
    x = np.meshgrid(np.arange(N, dtype=float), np.arange(ny, dtype=float))[0]
    phi = wl.tanh_profile(10.0 - np.abs(x - N / 2), 4.0)
    z = np.zeros((ny, N))
    s = _sim(p, dict(phi=phi, q=z, ux=z + u0, uy=z))

    def variance(t):
        q = s.fields()["phi"]
        d = (x - (N / 2 + u0 * t) + N / 2) % N - N / 2
        m = (q * d).sum() / q.sum()
        return (q * (d - m) ** 2).sum() / q.sum()

    s.step(t1)
    a = variance(t1)
    s.step(t2 - t1)
    return variance(t2) - a


def test_translated_band_keeps_its_profile():
    """The band carried by a uniform flow (u = 0.05) keeps its width: its variance
    changes by less than 0.02 over 200 steps (measured 0.002).  This pins the second-order
    time term 1/2 dt^2 d_t G of the CH evolution (Eq. weq45, the derivative a backward
    difference) with the advective forcing G of Eq. weq47."""
    assert abs(translated_band_spread_change()) < 0.02


def test_planted_mistake_ch_source_time_term_fails(monkeypatch):
    """Planted mistake: the 1/2 dt^2 d_t G term of Eq. weq45 left out (every step taken
    as the first, so G^n - G^(n-1) = 0).  The translated band then narrows: its variance
    falls by about 0.48 over the same 200 steps."""
    orig = ehd.Sim._one_step

    def wrong(self):
        self.history_valid = False
        return orig(self)

    monkeypatch.setattr(ehd.Sim, "_one_step", wrong)
    assert translated_band_spread_change() < -0.2


# ---------------------------------------------------------------------------------------
# Hydrodynamic LBE
# ---------------------------------------------------------------------------------------


def uniform_flow_errors(rho_l, phi0, steps=20, N=16, u=(0.06, -0.03), p0=0.01):
    """A single phase (phi = phi0 everywhere, so no interface, charge or force) moving at
    the uniform velocity u with the uniform pressure p0, periodic: the exact solution is
    that nothing changes.  Returns the largest deviations of u and p after `steps` steps."""
    p = wl.make_params(nx=N, ny=N, walls_y=0, rho_l=rho_l, rho_v=1.0, mu_l=0.1, mu_v=0.1,
                       eps_l=1.0, eps_v=1.0, sigma_l=0.0, sigma_v=0.0, alpha=0.02,
                       gamma=0.01, width=4.0, mobility=0.05, poisson_fixed_iter=1,
                       neutralize_charge=1)
    z = np.zeros((N, N))
    s = ehd.Sim(p)
    s.set_fields(z + phi0, z, z + u[0], z + u[1], z + p0)
    s.step(steps)
    F = s.fields()
    du = max(np.abs(F["ux"] - u[0]).max(), np.abs(F["uy"] - u[1]).max())
    return du, np.abs(F["p"] - p0).max()


@pytest.mark.parametrize("rho_l,phi0", [(1.0, 0.0), (3.0, 1.0)])
def test_uniform_flow_keeps_velocity_and_pressure(rho_l, phi0):
    """Uniform flow is an exact steady state (Galilean invariance): after 20 steps u and p
    equal their initial values to rounding (1e-14).  The pressure is the moment of
    Eq. eq32, whose rho s_0(u) term removes the velocity's share of the rest population."""
    du, dp = uniform_flow_errors(rho_l, phi0)
    assert du < 1e-14 and dp < 1e-14


def density_band_velocity_error(u0=0.05, N=64, steps=200, rho_ratio=3.0, width=8.0, axis="x"):
    """A band of the heavier phase (density ratio 3, 20 nodes wide, interfaces of width 8)
    carried by a uniform flow u0 across its interfaces, along `axis`, in a periodic box
    N long and 4 wide.  The exact solution translates everything unchanged, u = u0
    everywhere.  Returns the largest |u - u0| / u0 seen at four times over `steps` steps
    (inf if the run blows up)."""
    nx, ny = (N, 4) if axis == "x" else (4, N)
    p = wl.make_params(nx=nx, ny=ny, walls_y=0, rho_l=rho_ratio, rho_v=1.0, mu_l=0.1,
                       mu_v=0.1, eps_l=1.0, eps_v=1.0, sigma_l=0.0, sigma_v=0.0, alpha=0.02,
                       gamma=0.01, width=width, mobility=0.05, poisson_fixed_iter=1,
                       neutralize_charge=1)
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    s_coord = x if axis == "x" else y
    z = np.zeros((ny, nx))
    along, across = (z + u0, z) if axis == "x" else (z, z + u0)
    s = _sim(p, dict(phi=wl.tanh_profile(10.0 - np.abs(s_coord - N / 2), width), q=z,
                     ux=along, uy=across), z)
    key = "ux" if axis == "x" else "uy"
    worst = 0.0
    for _ in range(4):
        try:
            s.step(steps // 4)
        except FloatingPointError:
            return math.inf
        F = s.fields()
        other = "uy" if axis == "x" else "ux"
        worst = max(worst, np.abs(F[key] - u0).max() / u0, np.abs(F[other]).max() / u0)
    return worst


@pytest.mark.parametrize("axis", ["x", "y"])
def test_density_contrast_carried_by_uniform_flow(axis):
    """A density contrast moving with the flow, along either axis: u stays within 8 % of
    u0 (measured 3 %, of which 1.3 % is there without any contrast: the initial tanh
    profile is not the lattice's own equilibrium).  This pins the density-gradient parts
    of the hydrodynamic forcing (Eq. weq39) and of the pressure (Eq. eq32), which only act
    where density varies in a moving fluid, and that each axis uses its own gradient."""
    assert density_band_velocity_error(axis=axis) < 0.08


@pytest.mark.parametrize("mistake", ["forcing without its tensor term",
                                     "pressure without u.grad(rho)/2"])
def test_planted_mistakes_in_density_gradient_terms_fail(monkeypatch, mistake):
    """Planted mistakes: the u grad(rho):(c_i c_i - c_s^2 I)/c_s^2 part of R_bar_i
    (Eq. weq39) left out (u then strays by 20 %), or the (dt/2) u.grad(rho) part of the
    pressure (Eq. eq32) left out (the band's flow grows without bound)."""
    if mistake.startswith("forcing"):
        def wrong(P, ux, uy, grho_x, grho_y, Fx, Fy):
            out = np.empty((9,) + np.shape(ux))
            ug = ux * grho_x + uy * grho_y
            for i in range(9):
                out[i] = ehd.W[i] * (ug + (ehd.CX[i] * Fx + ehd.CY[i] * Fy) / ehd.CS2)
            return out

        monkeypatch.setattr(ehd, "f_force", wrong)
    else:
        orig = ehd.Sim._pressure

        def wrong(self, phi, rho, ux, uy, gphi_x, gphi_y):
            d = self.P.rho_l - self.P.rho_v
            return (orig(self, phi, rho, ux, uy, gphi_x, gphi_y) - ehd.CS2 / (1.0 - ehd.W[0])
                    * 0.5 * d * (ux * gphi_x + uy * gphi_y))

        monkeypatch.setattr(ehd.Sim, "_pressure", wrong)
    with np.errstate(all="ignore"):
        assert density_band_velocity_error() > 0.12


def test_planted_mistake_pressure_without_velocity_term_fails(monkeypatch):
    """Planted mistake: the rho s_0(u) term left out of the pressure moment (Eq. eq32).
    Each step then feeds the wrong pressure back into the equilibrium, and the uniform
    flow's pressure drifts away from p0 (by 0.047 after 20 steps here)."""
    orig = ehd.Sim._pressure

    def wrong(self, phi, rho, ux, uy, gphi_x, gphi_y):
        return (orig(self, phi, rho, ux, uy, gphi_x, gphi_y)
                - ehd.CS2 / (1.0 - ehd.W[0]) * rho * ehd.s_i(ux, uy)[0])

    monkeypatch.setattr(ehd.Sim, "_pressure", wrong)
    du, dp = uniform_flow_errors(1.0, 0.0)
    assert dp > 1e-2


def test_momentum_budget_exact():
    """Exact momentum budget of the hydro LBE on a fully periodic domain (Eqs. weq38,
    weq39 with sum c_i R_bar_i = F, and the lagged u closure of Algorithm 1): sum_x sum_i c f
    changes per step by sum_x [F^{n-1}/(2 tau_f) + (1 - 1/(2 tau_f)) F^n]."""
    N = 20
    p = wl.make_params(nx=N, ny=N, walls_y=0, rho_l=3.0, rho_v=1.0, mu_l=0.3, mu_v=0.05,
                       eps_l=5.0, eps_v=1.0, sigma_l=0.01, sigma_v=0.05, alpha=0.05,
                       gamma=0.01, width=4.0, neutralize_charge=1)
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    phi = wl.tanh_profile(5.0 - np.sqrt((x - 9.5) ** 2 + (y - 9.5) ** 2), 4.0)
    f = wl.perturbed(p, dict(phi=phi, q=0 * phi, ux=0 * phi, uy=0 * phi), seed=2)
    s = _sim(p, f)
    cx = ehd.CX[:, None, None]
    cy = ehd.CY[:, None, None]
    for _ in range(3):
        mx, my = (cx * s.f).sum(), (cy * s.f).sum()
        Fx_prev, Fy_prev = s.Fx_prev.copy(), s.Fy_prev.copy()
        phi_n = s.g.sum(0)
        s.step(1)
        tf = ehd.tau_f_of(s.P, phi_n)
        ex = np.sum(Fx_prev / (2 * tf) + (1 - 1 / (2 * tf)) * s.Fx_prev)
        ey = np.sum(Fy_prev / (2 * tf) + (1 - 1 / (2 * tf)) * s.Fy_prev)
        scale = np.abs(s.f).sum()
        assert abs((cx * s.f).sum() - mx - ex) < 1e-12 * scale
        assert abs((cy * s.f).sum() - my - ey) < 1e-12 * scale


def test_poiseuille_second_order():
    """Body-force-driven channel flow between half-way bounce-back walls: the steady
    parabola is kept to O(dx^2) (error falls ~4x per doubling)."""
    errs = []
    for ny in (16, 32):
        nu, g = 0.1, 1e-6
        p = wl.make_params(nx=4, ny=ny, walls_y=1, mu_l=nu, mu_v=nu, body_gx=g)
        z = np.zeros((ny, 4))
        ua = np.repeat(an.poiseuille(ny, g, nu)[:, None], 4, axis=1)
        s = _sim(p, dict(phi=z, q=z, ux=ua, uy=z))
        s.step(1500)
        errs.append(an.rel_l2(s.fields()["ux"], ua))
    assert errs[0] < 5e-3 and errs[0] / errs[1] > 3.5


def test_taylor_green_decay():
    """Taylor-Green vortex on a periodic grid decays as exp(-2 nu k^2 t) (textbook);
    measured amplitude decay rate within 2 %."""
    N, nu, U = 32, 0.05, 1e-3
    k = 2 * math.pi / N
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    ux = -U * np.cos(k * x) * np.sin(k * y)
    uy = U * np.sin(k * x) * np.cos(k * y)
    p0 = -U * U / 4 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    p = wl.make_params(nx=N, ny=N, walls_y=0, mu_l=nu, mu_v=nu)
    z = np.zeros((N, N))
    s = _sim(p, dict(phi=z, q=z, ux=ux, uy=uy), p0)
    t = 200
    s.step(t)
    F = s.fields()
    amp = math.sqrt((F["ux"] ** 2 + F["uy"] ** 2).mean() / (ux ** 2 + uy ** 2).mean())
    rate = -math.log(amp) / t
    assert abs(rate / (2 * nu * k * k) - 1.0) < 0.02


def test_laplace_law():
    """Static drop: the pressure jump equals gamma / r in two dimensions (Laplace law),
    measured as the time average over the drop's capillary ringing, within 10 %."""
    N, r, gamma = 48, 12, 0.03
    p = wl.make_params(nx=N, ny=N, walls_y=0, gamma=gamma, width=4.0, mobility=0.1,
                       mu_l=0.2, mu_v=0.2)
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    d = np.sqrt((x - (N - 1) / 2) ** 2 + (y - (N - 1) / 2) ** 2)
    phi0 = wl.tanh_profile(r - d, 4.0)
    z = np.zeros((N, N))
    s = _sim(p, dict(phi=phi0, q=z, ux=z, uy=z))
    s.step(600)
    jumps = []
    for _ in range(12):
        s.step(50)
        F = s.fields()
        inside = F["p"][d < r - 4].mean()
        outside = F["p"][d > r + 6].mean()
        jumps.append(inside - outside)
    assert abs(np.mean(jumps) / (gamma / r) - 1.0) < 0.1
