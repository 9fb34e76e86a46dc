"""Pins of the oracle's lattice, equilibria, source terms, stencils and streaming.

Each check is a property fixed by the mathematics (textbook D2Q9 isotropy, the exact
moment identities the paper states in its appendices, exactness of the stencils on
polynomials) rather than a retyped formula.
"""
import math

import numpy as np
import pytest

from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl

RNG = np.random.default_rng(1234)


def _P(**kw):
    base = dict(nx=5, ny=4, eps_v=0.7, eps_l=13.0, rho_l=3.0, rho_v=0.5, mu_l=0.2,
                mu_v=0.05, sigma_l=0.02, sigma_v=0.005, alpha=0.05)
    base.update(kw)
    return ehd.Params.from_dict(wl.make_params(**base))


def test_d2q9_isotropy():
    """sum w = 1, sum w c = 0, sum w c c = c_s^2 I, sum w c c c c = c_s^4 (dd + dd + dd):
    the D2Q9 lattice of Eq. weq37 with its weights is fourth-order isotropic."""
    c = ehd.C.astype(float)
    w = ehd.W
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2, np.eye(2) / 3.0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-15)
    # speeds 0, 1 (x4), sqrt 2 (x4) and opposite pairs
    assert sorted((c ** 2).sum(1).tolist()) == [0, 1, 1, 1, 1, 2, 2, 2, 2]
    assert np.array_equal(ehd.C[ehd.OPP], -ehd.C)
    assert abs(ehd.VARPI.sum() - 1.0) < 1e-15 and ehd.VARPI[0] == 0.0


def _moments(d):
    c = ehd.C.astype(float)
    m0 = d.sum(0)
    m1 = np.einsum("ia,i...->a...", c, d)
    m2 = np.einsum("ia,ib,i...->ab...", c, c, d)
    return m0, m1, m2


def test_h_eq_moments_eqA3():
    """Appendix A, Eq. eqA.3: sum h_eq = 0, sum c h_eq = 0, sum c c h_eq = c_s^2 varphi I;
    and Eq. weq55 recovers varphi from h_eq."""
    v = RNG.normal(size=(3, 4))
    h = ehd.h_eq(v)
    m0, m1, m2 = _moments(h)
    assert np.allclose(m0, 0, atol=1e-15)
    assert np.allclose(m1, 0, atol=1e-15)
    for a in range(2):
        for b in range(2):
            assert np.allclose(m2[a, b], (a == b) * v / 3.0, atol=1e-15)
    assert np.allclose(ehd.varphi_of(h), v, atol=1e-15)


def test_l_eq_moments_eqB1():
    """Appendix B, Eq. eqB.1: sum l_eq = q, sum c l_eq = q u, sum c c l_eq = c_s^2 q I."""
    q = RNG.normal(size=(3, 4))
    ux, uy = RNG.normal(size=(2, 3, 4)) * 0.05
    m0, m1, m2 = _moments(ehd.l_eq(q, ux, uy))
    assert np.allclose(m0, q, atol=1e-15)
    assert np.allclose(m1[0], q * ux, atol=1e-15) and np.allclose(m1[1], q * uy, atol=1e-15)
    for a in range(2):
        for b in range(2):
            assert np.allclose(m2[a, b], (a == b) * q / 3.0, atol=1e-15)


def test_g_eq_and_f_eq_moments():
    """sum g_eq = phi, sum c g_eq = 0, sum c c g_eq = c_s^2 hbar I (Eq. weq46);
    sum f_eq = 0, sum c f_eq = rho u, sum c c f_eq = p I + rho u u (Eq. weq40)."""
    P = _P()
    phi = RNG.uniform(0, 1, size=(3, 4))
    mu = RNG.normal(size=(3, 4)) * 1e-3
    m0, m1, m2 = _moments(ehd.g_eq(P, phi, mu))
    assert np.allclose(m0, phi, atol=1e-15) and np.allclose(m1, 0, atol=1e-16)
    assert np.allclose(m2[0, 0], mu / 3, atol=1e-16) and np.allclose(m2[0, 1], 0, atol=1e-16)
    p = RNG.normal(size=(3, 4)) * 1e-3
    rho = ehd.rho_of(P, phi)
    ux, uy = RNG.normal(size=(2, 3, 4)) * 0.05
    m0, m1, m2 = _moments(ehd.f_eq(P, p, rho, ux, uy))
    assert np.allclose(m0, 0, atol=1e-15)
    assert np.allclose(m1[0], rho * ux, atol=1e-15) and np.allclose(m1[1], rho * uy, atol=1e-15)
    assert np.allclose(m2[0, 0], p + rho * ux * ux, atol=1e-15)
    assert np.allclose(m2[1, 1], p + rho * uy * uy, atol=1e-15)
    assert np.allclose(m2[0, 1], rho * ux * uy, atol=1e-15)


def test_source_moments():
    """G_i (Eq. weq47): sum G = -u.grad phi, first and second moments 0.
    R_bar_i (Eq. weq39): sum R_bar = u.grad rho, sum c R_bar = F.
    Potential forcing (Eq. weq53): zero sum, first moment -eps_hat grad varphi / tau_h."""
    s = RNG.normal(size=(3, 4))
    m0, m1, m2 = _moments(ehd.g_source(s))
    assert np.allclose(m0, -s, atol=1e-15)
    assert np.allclose(m1, 0, atol=1e-15) and np.allclose(m2, 0, atol=1e-15)
    P = _P()
    ux, uy, gx, gy, Fx, Fy = RNG.normal(size=(6, 3, 4))
    m0, m1, _ = _moments(ehd.f_force(P, ux, uy, gx, gy, Fx, Fy))
    assert np.allclose(m0, ux * gx + uy * gy, atol=1e-14)
    assert np.allclose(m1[0], Fx, atol=1e-14) and np.allclose(m1[1], Fy, atol=1e-14)
    # potential collision: with q = 0 and h at equilibrium plus a first moment
    phi = RNG.uniform(0, 1, size=(3, 4))
    eh = ehd.eps_hat_of(P, phi)
    h = ehd.h_eq(RNG.normal(size=(3, 4))) + 0.01 * np.einsum(
        "i,i...->i...", ehd.W, RNG.normal(size=(9, 3, 4)))
    post = ehd.poisson_collide(P, h, eh, np.zeros((3, 4)))
    gvx, gvy = ehd.grad_varphi_local(P, h, eh)
    m0h, m1h, _ = _moments(h)
    m0p, m1p, _ = _moments(post)
    # zeroth moment relaxes toward sum h_eq = 0, first moment relaxes and is forced
    assert np.allclose(m0p, m0h - m0h / P.tau_h, atol=1e-15)
    assert np.allclose(m1p[0], m1h[0] * (1 - 1 / P.tau_h) - eh * gvx / P.tau_h, atol=1e-15)
    assert np.allclose(m1p[1], m1h[1] * (1 - 1 / P.tau_h) - eh * gvy / P.tau_h, atol=1e-15)


def test_local_gradient_is_consistent_first_moment():
    """Eq. eqA.16 solved for the first moment: after one forced collision the first moment
    is -(eps_hat + c_s^2 tau_h) grad varphi scaled by (1 - c_s^2/(eps_hat + c_s^2 tau_h)),
    i.e. the forcing turns the first-moment relaxation time into tau_h + eps_hat/c_s^2, the
    relaxation time of a plain diffusion LBE with diffusivity eps(phi)."""
    P = _P()
    phi = RNG.uniform(0, 1, size=(3, 4))
    eh = ehd.eps_hat_of(P, phi)
    h = ehd.h_eq(np.zeros((3, 4))) + 0.01 * RNG.normal(size=(9, 3, 4))
    post = ehd.poisson_collide(P, h, eh, np.zeros((3, 4)))
    _, m1h, _ = _moments(h)
    _, m1p, _ = _moments(post)
    tau_eff = P.tau_h + eh / ehd.CS2
    assert np.allclose(m1p, m1h * (1 - 1 / tau_eff), atol=1e-15)
    # and the diffusivity of that relaxation time is eps(phi) (Eq. eqA.15 with eps)
    assert np.allclose(ehd.CS2 * (tau_eff - 0.5), ehd.eps_of(P, phi), atol=1e-14)


def test_property_laws():
    """Remark II: eps(0) = eps_v, eps(1) = eps_l, eps'(0) = eps'(1) = 0 (reduction
    consistency); eps' is the derivative of eps (checked by central differences);
    linear laws hit both phase values."""
    P = _P()
    assert ehd.eps_of(P, 0.0) == P.eps_v and abs(ehd.eps_of(P, 1.0) - P.eps_l) < 1e-14
    assert ehd.deps_dphi(P, 0.0) == 0.0 and ehd.deps_dphi(P, 1.0) == 0.0
    x = np.linspace(0.05, 0.95, 19)
    d = 1e-6
    fd = (ehd.eps_of(P, x + d) - ehd.eps_of(P, x - d)) / (2 * d)
    assert np.allclose(fd, ehd.deps_dphi(P, x), rtol=1e-8)
    assert np.allclose(ehd.eps_hat_of(P, x), ehd.eps_of(P, x) - P.eps_v, atol=1e-14)
    for fn, a, b in ((ehd.rho_of, P.rho_v, P.rho_l), (ehd.mu_of, P.mu_v, P.mu_l),
                     (ehd.sigma_of, P.sigma_v, P.sigma_l)):
        assert abs(fn(P, 0.0) - a) < 1e-15 and abs(fn(P, 1.0) - b) < 1e-15
    # viscosity law (Sec. 3.1): mu = rho c_s^2 (tau_f - 1/2)
    assert np.allclose(ehd.rho_of(P, x) / 3 * (ehd.tau_f_of(P, x) - 0.5), ehd.mu_of(P, x))


def test_stencils_exact_on_quadratics():
    """The isotropic stencils (Sec. 3.2) are exact on quadratic polynomials: on
    T = a x^2 + b x y + c y^2 + d x + e y, grad T and lap T = 2a + 2c are reproduced at
    every node whose 3x3 neighbourhood lies in the field."""
    P = _P(nx=9, ny=8, walls_y=0)
    y, x = np.meshgrid(np.arange(8.0), np.arange(9.0), indexing="ij")
    a, b, c, d, e = 0.3, -0.7, 0.11, 0.5, -1.3
    T = a * x * x + b * x * y + c * y * y + d * x + e * y
    ext = ehd.extend_with_ghosts(P, T, 0.0, 0.0)
    gx, gy = ehd.gradient(ext)
    lap = ehd.laplacian(ext)
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(gx[inner], (2 * a * x + b * y + d)[inner], atol=1e-12)
    assert np.allclose(gy[inner], (b * x + 2 * c * y + e)[inner], atol=1e-12)
    assert np.allclose(lap[inner], 2 * a + 2 * c, atol=1e-12)


def test_stencils_second_order_and_telescoping():
    """On a periodic sine the stencil errors fall by 4x per grid doubling, and the periodic
    gradient sums to zero (telescoping)."""
    errs = []
    for N in (16, 32, 64):
        P = _P(nx=N, ny=N, walls_y=0)
        k = 2 * math.pi / N
        y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float),
                           indexing="ij")
        T = np.sin(k * x + 0.3) * np.cos(2 * k * y)
        ext = ehd.extend_with_ghosts(P, T, 0.0, 0.0)
        gx, gy = ehd.gradient(ext)
        lap = ehd.laplacian(ext)
        ex_gx = k * np.cos(k * x + 0.3) * np.cos(2 * k * y)
        ex_lap = -5 * k * k * T
        errs.append((np.abs(gx - ex_gx).max() / k, np.abs(lap - ex_lap).max() / (5 * k * k)))
        assert abs(gx.sum()) < 1e-12 and abs(gy.sum()) < 1e-12
    for j in range(2):
        r1 = errs[0][j] / errs[1][j]
        r2 = errs[1][j] / errs[2][j]
        assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2


def test_wetting_ghost_rows():
    """Eq. weq68 with sqrt(2 beta/kappa) = 4/W: theta = 90 deg gives a zero normal
    gradient (mirror); theta < 90 raises the ghost value where 0 < phi < 1 (phase l wets
    the wall); the top wall mirrors the bottom one."""
    P = _P(nx=6, ny=5, walls_y=1, width=4.0)
    phi = RNG.uniform(0.05, 0.95, size=(5, 6))
    ext = ehd.extend_with_ghosts(P, phi, 0.0, 0.0)
    assert np.allclose(ext[0, 1:-1], phi[0]) and np.allclose(ext[-1, 1:-1], phi[-1])
    ext = ehd.extend_with_ghosts(P, phi, 1.0, 1.0)
    assert math.isclose(math.sqrt(2 * P.beta / P.kappa), 4.0 / P.width, rel_tol=1e-14)
    # one-sided normal derivative across each wall equals -(4/W) cos(theta) (phi - phi^2)
    dn_bottom = phi[0] - ext[0, 1:-1]
    dn_top = phi[-1] - ext[-1, 1:-1]
    assert np.allclose(dn_bottom, -(4 / P.width) * (phi[0] - phi[0] ** 2))
    assert np.allclose(dn_top, -(4 / P.width) * (phi[-1] - phi[-1] ** 2))
    # periodic x frame including the ghost rows
    assert np.allclose(ext[:, 0], ext[:, -2]) and np.allclose(ext[:, -1], ext[:, 1])


@pytest.mark.parametrize("walls", [0, 1])
def test_streaming_moves_along_c(walls):
    """A unit population i at node (x, y) sits at (x + c_i, y + c_i) after streaming (pull
    form of f_i(x + c_i, t + 1) = f*_i(x, t)); at a wall it returns in the opposite
    direction at the same node; bounce-back streaming conserves the total."""
    P = _P(nx=5, ny=4, walls_y=walls)
    for i in range(9):
        for (x, y) in ((2, 1), (0, 0), (4, 3)):
            post = np.zeros((9, 4, 5))
            post[i, y, x] = 1.0
            new = ehd.stream(P, post, "bb")
            cx, cy = ehd.C[i]
            ty = y + cy
            if walls and not (0 <= ty < 4):
                assert new[ehd.OPP[i], y, x] == 1.0 and new.sum() == 1.0
            else:
                assert new[i, ty % 4, (x + cx) % 5] == 1.0 and new.sum() == 1.0
    post = RNG.normal(size=(9, 4, 5))
    assert abs(ehd.stream(P, post, "bb").sum() - post.sum()) < 1e-12


def test_anti_bounce_back_dirichlet():
    """Anti-bounce-back: a population entering from a wall is -h*_opp + 2 w_i varphi_w, so
    an equilibrium of a potential equal to the wall value is left unchanged there."""
    P = _P(nx=5, ny=4, walls_y=1)
    v = np.full((4, 5), 0.37)
    new = ehd.stream(P, ehd.h_eq(v), "abb", (0.37, 0.37))
    assert np.allclose(new, ehd.h_eq(v), atol=1e-15)


def test_set_fields_reproduces_inputs():
    """Algorithm 1 step 1: right after initialisation the moments of the populations are
    the given fields (phi, q, u, p) exactly."""
    p, f = wl.planar_layers(nx=5, ny=12, varphi_high=0.05)
    f = wl.perturbed(p, f, seed=3)
    p0 = RNG.normal(size=(12, 5)) * 1e-4
    sim = ehd.Sim(p)
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"], p0)
    F = sim.fields()
    for k in ("phi", "q", "ux", "uy"):
        assert np.allclose(F[k], f[k], atol=1e-14, rtol=0), k
    assert np.allclose(F["p"], p0, atol=1e-10)


def test_charge_source_is_minus_div_sigma_E():
    """With Gauss's law q = div(eps E) (Eq. weq32), the source of Eq. weq57 equals
    -div(sigma E), the divergence of the ohmic current (checked with analytic fields:
    phi(x, y), E = -grad v for a smooth v, exact derivatives)."""
    P = _P()
    x, y = np.meshgrid(np.linspace(0, 1, 7), np.linspace(0, 1, 6))
    phi = 0.5 + 0.4 * np.sin(2 * x + y)
    phx, phy = 0.8 * np.cos(2 * x + y), 0.4 * np.cos(2 * x + y)
    # v = x^2 y + cos(y): E = -(2xy, x^2 - sin y), div E = -(2y - cos y)
    Ex, Ey = -2 * x * y, -(x * x - np.sin(y))
    divE = -(2 * y - np.cos(y))
    eps, de = ehd.eps_of(P, phi), ehd.deps_dphi(P, phi)
    sig, ds = ehd.sigma_of(P, phi), P.sigma_l - P.sigma_v
    q = eps * divE + de * (phx * Ex + phy * Ey)
    div_sigma_E = sig * divE + ds * (phx * Ex + phy * Ey)
    R = ehd.charge_source(P, phi, q, phx, phy, Ex, Ey)
    assert np.allclose(R, -div_sigma_E, rtol=1e-12, atol=1e-14)


def test_electric_chemical_potential_is_variational():
    """The electric part of hbar is the phi-derivative of the field energy |D|^2 / (2 eps)
    at fixed displacement D (Eq. weq17): -eps' |D|^2 / (2 eps^2) = -eps' |E|^2 / 2."""
    P = _P()
    phi = np.linspace(0.05, 0.95, 10)
    Ex, Ey = 0.3, -0.2
    Dx, Dy = ehd.eps_of(P, phi) * Ex, ehd.eps_of(P, phi) * Ey
    d = 1e-6
    energy = lambda ph: (Dx * Dx + Dy * Dy) / (2 * ehd.eps_of(P, ph))
    fd = (energy(phi + d) - energy(phi - d)) / (2 * d)
    z = np.zeros_like(phi)
    electric = ehd.chemical_potential(P, phi, z, Ex, Ey) - ehd.chemical_potential(P, phi, z, 0.0, 0.0)
    assert np.allclose(electric, fd, rtol=1e-7)
    # the bulk part is d/dphi of beta phi^2 (phi - 1)^2 (Sec. 2.2)
    bulk = ehd.chemical_potential(P, phi, z, 0.0, 0.0)
    psi = lambda ph: P.beta * ph ** 2 * (ph - 1) ** 2
    assert np.allclose(bulk, (psi(phi + d) - psi(phi - d)) / (2 * d), rtol=1e-7)


def test_fields_mu_flat_interface_at_rest_is_near_zero():
    """The output chemical potential of a flat tanh interface with no field: the profile
    0.5 + 0.5 tanh(2 y / W) makes the bulk term 4 beta phi (phi - 1/2)(phi - 1) and
    kappa lap(phi) cancel exactly in the continuum (Sec. 2.2), so the discrete hbar is
    O(1/W^2) of either term (second order: doubling W divides it by about four); a
    dropped kappa term or a wrong sign leaves it O(1)."""
    ratios = []
    for W in (8.0, 16.0):
        P0, f = wl.planar_layers(nx=4, ny=int(12 * W), varphi_high=0.0, width=W)
        sim = ehd.Sim(P0)
        sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        F = sim.fields()
        P = sim.P
        phi = F["phi"]
        bulk = 4.0 * P.beta * phi * (phi - 0.5) * (phi - 1.0)
        assert np.abs(bulk).max() > 1e-3 * P.beta
        ratios.append(np.abs(F["mu"]).max() / np.abs(bulk).max())
    assert ratios[0] < 0.05
    assert 3.5 < ratios[0] / ratios[1] < 4.5


def test_fields_mu_uniform_phase_in_uniform_field():
    """A uniform phase phi = c between electrodes: eps is uniform, the potential is linear
    and E = (varphi_b - varphi_t) / ny everywhere, the Laplacian of phi vanishes (90 degree
    walls), so hbar = 4 beta c (c - 1/2)(c - 1) - eps'(c) E^2 / 2 exactly (Eq. weq31).
    (A fixed, long potential loop: the linear start already has the right potential, so
    the relative-change rule would stop before the first moment, which carries E, has
    developed.)"""
    c, vb = 0.3, 0.2
    P0 = wl.make_params(nx=3, ny=20, walls_y=1, eps_l=6.0, eps_v=1.0, sigma_l=0.0,
                        sigma_v=0.0, gamma=0.01, width=4.0, varphi_bottom=vb, varphi_top=0.0,
                        poisson_fixed_iter=6000)
    z = np.zeros((20, 3))
    sim = ehd.Sim(P0)
    sim.set_fields(z + c, z, z, z)
    F = sim.fields()
    P = sim.P
    E = vb / 20.0
    assert np.allclose(F["Ey"], E, rtol=1e-6, atol=0)
    want = 4.0 * P.beta * c * (c - 0.5) * (c - 1.0) - 0.5 * ehd.deps_dphi(P, c) * E * E
    field_part = 0.5 * ehd.deps_dphi(P, c) * E * E
    assert abs(field_part) > 1e-3 * abs(want)
    assert np.allclose(F["mu"], want, rtol=0, atol=1e-6 * abs(field_part))


def test_initial_ch_populations_carry_the_initial_chemical_potential():
    """Algorithm 1 step 1 (reading R12): the CH populations start at the equilibrium of
    Eq. weq46 for the initial phi and its chemical potential (Eq. weq31, no field yet).
    That equilibrium's second moment is c_s^2 hbar I, so sum_i c_iy^2 g_i = c_s^2 hbar,
    sum_i c_ix c_iy g_i = 0 and sum_i g_i = phi.  hbar is formed here from the bulk term
    and kappa times the central second difference, which is the isotropic Laplacian for a
    profile along y (a periodic band, so no wall rows)."""
    ny, nx = 32, 4
    p = wl.make_params(nx=nx, ny=ny, walls_y=0)
    P = ehd.Params.from_dict(p)
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    # a band twice as steep as the equilibrium profile, so that hbar is far from zero
    phi = wl.tanh_profile(8.0 - np.abs(y - ny / 2), 0.5 * p["width"])
    z = np.zeros((ny, nx))
    s = ehd.Sim(p)
    s.set_fields(phi, z, z, z)
    lap = np.roll(phi, 1, axis=0) + np.roll(phi, -1, axis=0) - 2.0 * phi
    hbar = 4.0 * P.beta * phi * (phi - 0.5) * (phi - 1.0) - P.kappa * lap
    cx = np.array([c[0] for c in ehd.C], dtype=float)[:, None, None]
    cy = np.array([c[1] for c in ehd.C], dtype=float)[:, None, None]
    assert np.allclose((cy * cy * s.g).sum(axis=0), ehd.CS2 * hbar, atol=1e-14, rtol=0)
    assert np.allclose((cx * cy * s.g).sum(axis=0), 0.0, atol=1e-15)
    assert np.allclose(s.g.sum(axis=0), phi, atol=1e-14, rtol=0)
    assert np.abs(hbar).max() > 1e-3   # the check has something to see


def test_initial_populations_carry_the_initial_flux_and_momentum():
    """Algorithm 1 step 1 (reading R12): the charge and hydrodynamic populations start at
    the equilibria of Eqs. weq61 and weq40 for the initial fields, whose first moments are
    the charge flux q u and the momentum rho u (rho from the initial phi)."""
    ny, nx = 12, 10
    p = wl.make_params(nx=nx, ny=ny, walls_y=1, rho_l=3.0, rho_v=1.0)
    P = ehd.Params.from_dict(p)
    phi = RNG.uniform(0.0, 1.0, size=(ny, nx))
    q = RNG.normal(size=(ny, nx)) * 1e-3
    ux, uy = RNG.normal(size=(2, ny, nx)) * 1e-2
    s = ehd.Sim(p)
    s.set_fields(phi, q, ux, uy, RNG.normal(size=(ny, nx)) * 1e-3)
    cx = np.array([c[0] for c in ehd.C], dtype=float)[:, None, None]
    cy = np.array([c[1] for c in ehd.C], dtype=float)[:, None, None]
    rho = P.rho_v + phi * (P.rho_l - P.rho_v)
    assert np.allclose((cx * s.l).sum(axis=0), q * ux, atol=1e-16, rtol=0)
    assert np.allclose((cy * s.l).sum(axis=0), q * uy, atol=1e-16, rtol=0)
    assert np.allclose((cx * s.f).sum(axis=0), rho * ux, atol=1e-15, rtol=0)
    assert np.allclose((cy * s.f).sum(axis=0), rho * uy, atol=1e-15, rtol=0)
