"""Seeded synthetic workloads: parameter sets (lattice units) and initial fields.

This module holds no arithmetic of the lattice Boltzmann method itself.  It only
states problem set-ups: domain sizes, fluid properties, wall conditions and initial
fields (phi0, q0, ux0, uy0), all from fixed seeds.  The tests, the benchmark and the
CPU reference harness take their inputs from here, so the CUDA path and the CPU
oracle see identical inputs.

Set-ups (sizes and ratios follow the paper's workloads; the paper's datasets are not
needed, every input is generated):

* planar_layers      two superimposed fluids between electrodes (Sec. 6.1)
* gaussian_bell      single-phase charge relaxation of a Gaussian bell (Sec. 6.2)
* droplet            leaky-dielectric droplet in a uniform field (Sec. 7.1, Table 1)
* sessile_drop       sessile drop on an electrode with (reversed) electrowetting
                     (Sec. 6.3, Sec. 7.2)
* served_requests    a stream of droplet requests of mixed grid sizes
"""
from __future__ import annotations

import math

import numpy as np

# Keys of a parameter set; the same names are used by the C struct ehd_params.
PARAM_DEFAULTS = dict(
    nx=0, ny=0, walls_y=1, precision=0,
    rho_l=1.0, rho_v=1.0, mu_l=0.1, mu_v=0.1,
    sigma_l=0.0, sigma_v=0.0, eps_l=1.0, eps_v=1.0, alpha=0.1,
    gamma=0.01, width=4.0, mobility=0.1,
    theta_bottom_deg=90.0, theta_top_deg=90.0, ew_bottom=0.0, ew_sign=1.0,
    varphi_bottom=0.0, varphi_top=0.0, ramp_steps=0, neutralize_charge=0,
    body_gx=0.0, body_gy=0.0,
    poisson_tol=1e-5, poisson_max_iter=100000, poisson_min_iter=1, poisson_fixed_iter=0,
    poisson_loop=0, start_step=0, tile_rows=0, potential_scheme=0, chi=1.0, field_mode=0,
    lagged_field=0,
)


def make_params(**kw):
    p = dict(PARAM_DEFAULTS)
    for k, v in kw.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def _grid(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def tanh_profile(signed_distance, width):
    """Diffuse-interface initial profile 0.5 + 0.5 tanh(2 d / W) (the paper's initial
    condition, Sec. 6.3), d > 0 inside phase l."""
    return 0.5 + 0.5 * np.tanh(2.0 * signed_distance / width)


def smooth_random_field(nx, ny, rng, amplitude, modes=3, periodic_y=False):
    """Sum of a few low Fourier modes with seeded random amplitudes and phases.
    With walls in y the field is multiplied by a bump that vanishes at the walls."""
    x, y = _grid(nx, ny)
    out = np.zeros((ny, nx))
    for _ in range(modes):
        kx = rng.integers(1, 3)
        ky = rng.integers(1, 3)
        a = rng.uniform(-1.0, 1.0)
        px, py = rng.uniform(0, 2 * math.pi, size=2)
        out += a * np.sin(2 * math.pi * kx * x / nx + px) * np.sin(2 * math.pi * ky * y / ny + py)
    if not periodic_y:
        out *= np.sin(math.pi * (y + 0.5) / ny) ** 2
    m = np.abs(out).max()
    return amplitude * out / (m if m > 0 else 1.0)


# -------------------------------------------------------------------------------------
# Sec. 6.1: two superimposed planar fluids
# -------------------------------------------------------------------------------------


def planar_layers(nx=4, ny=64, eps_ratio=10.0, sigma_ratio=0.1, varphi_high=0.1,
                  eps_v=0.1, sigma_v=0.01, alpha=0.01, width=4.0, **over):
    """Fluid l (phi = 1) in the lower half, fluid v in the upper half, tanh interface at
    mid-height; high potential on the bottom wall, 0 on the top wall."""
    params = make_params(
        nx=nx, ny=ny, walls_y=1, rho_l=1.0, rho_v=1.0, mu_l=0.1, mu_v=0.1,
        eps_v=eps_v, eps_l=eps_ratio * eps_v, sigma_v=sigma_v, sigma_l=sigma_ratio * sigma_v,
        alpha=alpha, gamma=0.01, width=width, mobility=0.1,
        varphi_bottom=varphi_high, varphi_top=0.0)
    params.update(over)
    x, y = _grid(nx, ny)
    yc = (ny - 1) / 2.0
    phi0 = tanh_profile(yc - y, width)
    z = np.zeros((ny, nx))
    return params, dict(phi=phi0, q=z.copy(), ux=z.copy(), uy=z.copy())


# -------------------------------------------------------------------------------------
# Sec. 6.2: charge relaxation of a Gaussian bell
# -------------------------------------------------------------------------------------


def gaussian_bell(N, alpha=0.1, eps=1.0, potential_scale=1e-3, **over):
    """Single phase (phi = 0), periodic N x N, q0 = A exp(-r^2 / (2 s0^2)) with s0 = N/16,
    centred on node (N/2, N/2).  Diffusive scaling: the run lasts n = N^2 / (512 alpha)
    steps so that the bell's variance doubles; sigma/eps = 1/n so the total relaxation is
    e^{-1}.

    The amplitude A = potential_scale * eps / s0^2 keeps the bell's own potential near
    potential_scale: with uniform sigma and eps the charge equation is linear in q, so the
    relative error does not depend on A, while an O(1) charge in lattice units would drive
    the fluid with a body force q E far outside the incompressible flow model's range.
    Returns (params, fields, n_steps, s0)."""
    n_steps = int(round(N * N / (512.0 * alpha)))
    sigma = eps / n_steps
    params = make_params(
        nx=N, ny=N, walls_y=0, rho_l=1.0, rho_v=1.0, mu_l=0.1, mu_v=0.1,
        eps_l=eps, eps_v=eps, sigma_l=sigma, sigma_v=sigma, alpha=alpha,
        gamma=0.01, width=4.0, mobility=0.1, neutralize_charge=1)
    params.update(over)
    x, y = _grid(N, N)
    s0 = N / 16.0
    r2 = (x - N / 2) ** 2 + (y - N / 2) ** 2
    q0 = potential_scale * eps / (s0 * s0) * np.exp(-r2 / (2.0 * s0 * s0))
    z = np.zeros((N, N))
    return params, dict(phi=z.copy(), q=q0, ux=z.copy(), uy=z.copy()), n_steps, s0


# -------------------------------------------------------------------------------------
# Sec. 7.1: leaky-dielectric droplet in a uniform field
# -------------------------------------------------------------------------------------


def droplet_ratios(seed):
    """(R, S, Ca_E): conductivity and permittivity ratios (droplet / surrounding, the
    paper's meaning, Sec. 7.1) log-uniform on [0.1, 10]; Ca_E uniform on [0.05, 0.3]."""
    rng = np.random.default_rng(seed)
    R = float(10.0 ** rng.uniform(-1.0, 1.0))
    S = float(10.0 ** rng.uniform(-1.0, 1.0))
    Ca = float(rng.uniform(0.05, 0.3))
    return R, S, Ca


def droplet(seed=0, N=256, r=None, R=None, S=None, Ca=None, Re=1.0, Re_E=1e-3,
            rho_ratio=1.0, mu_ratio=1.0, gamma=1e-3, width=5.0, mobility=0.1, eps_v=1.0,
            alpha=0.01, **over):
    """Droplet (phase l) of radius r (default 40/256 of N) centred in an N x N box,
    periodic in x, electrodes at the bottom (0) and top (high) walls.

    Mapping of the dimensionless groups (Sec. 7.1) to lattice parameters:
    E0 = sqrt(Ca_E gamma / (eps_v r)); wall potential difference E0 * N;
    mu_v from Re = r^2 rho_v eps_v E0^2 / mu_v^2; sigma_v from
    Re_E = eps_v^2 E0^2 / (mu_v sigma_v), capped so that sigma/eps <= 0.25 in both fluids.
    Returns (params, fields, info)."""
    if R is None or S is None or Ca is None:
        R0, S0, Ca0 = droplet_ratios(seed)
        R = R0 if R is None else R
        S = S0 if S is None else S
        Ca = Ca0 if Ca is None else Ca
    if r is None:
        r = 40.0 * N / 256.0
    rho_v = 1.0
    E0 = math.sqrt(Ca * gamma / (eps_v * r))
    mu_v = math.sqrt(r * r * rho_v * eps_v * E0 * E0 / Re)
    sigma_re = eps_v * eps_v * E0 * E0 / (mu_v * Re_E)
    sigma_v = eps_v * min(0.25 / max(1.0, R / S), sigma_re)
    params = make_params(
        nx=N, ny=N, walls_y=1, rho_v=rho_v, rho_l=rho_ratio * rho_v, mu_v=mu_v,
        mu_l=mu_ratio * mu_v, eps_v=eps_v, eps_l=S * eps_v, sigma_v=sigma_v,
        sigma_l=R * sigma_v, alpha=alpha, gamma=gamma, width=width, mobility=mobility,
        varphi_bottom=0.0, varphi_top=E0 * N)
    params.update(over)
    x, y = _grid(N, N)
    d = np.sqrt((x - (N - 1) / 2.0) ** 2 + (y - (N - 1) / 2.0) ** 2)
    phi0 = tanh_profile(r - d, width)
    z = np.zeros((N, N))
    info = dict(R=R, S=S, Ca=Ca, E0=E0, r=r, Re_E_used=eps_v ** 2 * E0 ** 2 / (mu_v * sigma_v))
    return params, dict(phi=phi0, q=z.copy(), ux=z.copy(), uy=z.copy()), info


# -------------------------------------------------------------------------------------
# Sec. 6.3 / Sec. 7.2: sessile drop on an electrode, (reversed) electrowetting
# -------------------------------------------------------------------------------------


def sessile_drop(seed=0, nx=512, ny=1024, r=80.0, theta=None, rho_ratio=10.0,
                 mu_ratio=10.0, eps_ratio=20.0, ew=0.4, ew_sign=-1.0, voltage=0.5,
                 ramp_steps=20000, start_step=0, width=4.0, gamma=0.01, mobility=0.05,
                 **over):
    """Half-drop (phase l) of radius r centred on the bottom wall of an nx x ny box,
    periodic in x.  Contact angle theta ~ U[60, 120] degrees from the seed.  The top wall
    potential ramps linearly from 0 to `voltage` over ramp_steps; the bottom electrode is
    at 0.  Reversed electrowetting (ew_sign = -1) by default.  The surrounding fluid
    conducts (sigma_v = 0.02), the drop barely does (sigma_l = sigma_v / 100)."""
    rng = np.random.default_rng(seed)
    if theta is None:
        theta = float(rng.uniform(60.0, 120.0))
    rho_v = 1.0
    mu_v = 0.05
    eps_v = 1.0
    sigma_v = 0.02
    params = make_params(
        nx=nx, ny=ny, walls_y=1, rho_v=rho_v, rho_l=rho_ratio * rho_v, mu_v=mu_v,
        mu_l=mu_ratio * mu_v, eps_v=eps_v, eps_l=eps_ratio * eps_v, sigma_v=sigma_v,
        sigma_l=sigma_v / 100.0, alpha=0.01, gamma=gamma, width=width, mobility=mobility,
        theta_bottom_deg=theta, theta_top_deg=90.0, ew_bottom=ew, ew_sign=ew_sign,
        varphi_bottom=0.0, varphi_top=voltage, ramp_steps=ramp_steps,
        start_step=start_step)
    params.update(over)
    x, y = _grid(nx, ny)
    d = np.sqrt((x - (nx - 1) / 2.0) ** 2 + (y + 0.5) ** 2)
    phi0 = tanh_profile(r - d, width)
    z = np.zeros((ny, nx))
    return params, dict(phi=phi0, q=z.copy(), ux=z.copy(), uy=z.copy()), dict(theta=theta)


# -------------------------------------------------------------------------------------
# Perturbations used by the parity tests: exercise every term (flow, charge, history)
# -------------------------------------------------------------------------------------


def perturbed(params, fields, seed, u_amp=2e-3, q_amp=1e-3):
    """Adds a smooth seeded velocity field and a smooth seeded charge to a set-up so that
    every coupling term of the step is non-zero."""
    rng = np.random.default_rng(seed)
    ny, nx = fields["phi"].shape
    periodic_y = not params["walls_y"]
    out = dict(fields)
    out["ux"] = fields["ux"] + smooth_random_field(nx, ny, rng, u_amp, periodic_y=periodic_y)
    out["uy"] = fields["uy"] + smooth_random_field(nx, ny, rng, u_amp, periodic_y=periodic_y)
    out["q"] = fields["q"] + smooth_random_field(nx, ny, rng, q_amp, periodic_y=periodic_y)
    return out
