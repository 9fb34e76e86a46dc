"""Closed-form and quadrature solutions used to pin the oracle.

Each function states the problem it solves and where it comes from; none of them calls
the oracle or the CUDA path.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def rel_l2(num, ana):
    """Relative L2 error over the whole domain, the paper's error norm (Sec. 6.1)."""
    num = np.asarray(num, dtype=np.float64)
    ana = np.asarray(ana, dtype=np.float64)
    return float(np.sqrt(np.sum((num - ana) ** 2) / np.sum(ana ** 2)))


def fitted_order(ns, errs):
    """Least-squares slope of log(err) against log(1/n)."""
    a = np.polyfit(np.log(1.0 / np.asarray(ns, float)), np.log(np.asarray(errs, float)), 1)
    return float(a[0])


# -- Sec. 6.1: planar layers ----------------------------------------------------------


def planar_sharp(ny, R_hat, varphi_high):
    """Eq. weq72 on the lattice rows: walls at y = -1/2 and ny - 1/2, the lower fluid
    (conductivity ratio R_hat = sigma_lower / sigma_upper) below mid-height, potential
    varphi_high at the bottom and 0 at the top.  In units of the height:
    varphi_1 = (-2Y + R)/(1 + R) (lower), varphi_2 = R (1 - 2Y)/(1 + R) (upper)."""
    y = np.arange(ny, dtype=np.float64)
    Y = (y + 0.5) / ny - 0.5
    lower = (-2.0 * Y + R_hat) / (1.0 + R_hat)
    upper = (-2.0 * Y + 1.0) * R_hat / (1.0 + R_hat)
    return varphi_high * np.where(Y < 0.0, lower, upper)


def planar_diffuse(ny, phi_of_y, dphi_dy, sigma_of, eps_of, deps_dphi, dsigma_dphi,
                   varphi_bottom, varphi_top):
    """Steady 1-D potential and charge for a diffuse layer profile phi(y) with no flow
    and vanishing charge diffusion: the conduction current J = sigma E is uniform, so
    E(y) = J / sigma(y), J = (varphi_bottom - varphi_top) / int dy / sigma, and Gauss's law
    gives q = d(eps E)/dy = J d(eps/sigma)/dy.  Walls at y = -1/2 and ny - 1/2.
    Returns (varphi, q, E) at the lattice rows; the integrals use adaptive quadrature."""
    y0, y1 = -0.5, ny - 0.5
    inv_sigma = lambda s: 1.0 / sigma_of(phi_of_y(s))
    total, _ = integrate.quad(inv_sigma, y0, y1, limit=400, epsabs=1e-14, epsrel=1e-13)
    J = (varphi_bottom - varphi_top) / total
    ys = np.arange(ny, dtype=np.float64)
    varphi = np.empty(ny)
    q = np.empty(ny)
    E = np.empty(ny)
    for j, yj in enumerate(ys):
        part, _ = integrate.quad(inv_sigma, y0, yj, limit=400, epsabs=1e-14, epsrel=1e-13)
        varphi[j] = varphi_bottom - J * part
        ph = phi_of_y(yj)
        s = sigma_of(ph)
        e = eps_of(ph)
        dph = dphi_dy(yj)
        d_eps_over_sigma = (deps_dphi(ph) * s - e * dsigma_dphi(ph)) / (s * s) * dph
        q[j] = J * d_eps_over_sigma
        E[j] = J / s
    return varphi, q, E


# -- Sec. 6.2: Gaussian bell ----------------------------------------------------------


def gaussian_bell(N, t, s0, amplitude, alpha, sigma, eps):
    """Charge of a Gaussian bell under diffusion alpha and ohmic relaxation sigma/eps in
    an unbounded plane: q = A (s0^2/s^2) exp(-r^2/(2 s^2)) exp(-sigma t/eps),
    s^2 = s0^2 + 2 alpha t.  Eq. weq78 is the alpha -> 0 limit (with the exponent's sign
    taken as a decay).  Centre at node (N/2, N/2); periodic images are below 1e-13 for
    s <= N/11."""
    y, x = np.meshgrid(np.arange(N, dtype=np.float64), np.arange(N, dtype=np.float64),
                       indexing="ij")
    r2 = (x - N / 2) ** 2 + (y - N / 2) ** 2
    s2 = s0 * s0 + 2.0 * alpha * t
    return amplitude * (s0 * s0 / s2) * np.exp(-r2 / (2.0 * s2)) * math.exp(-sigma * t / eps)


# -- Sec. 7.1: small-deformation theories ---------------------------------------------


def taylor_D(R, S, Ca, B=1.0):
    """Taylor's small-deformation result, Eq. eq53 (R conductivity, S permittivity,
    B viscosity ratio)."""
    return 9.0 / 16.0 * Ca / (2.0 + R) ** 2 * (R * R + 1.0 - 2.0 * S
                                             + 0.6 * (R - S) * (2.0 + 3.0 * B) / (1.0 + B))


def feng_D(R, S, Ca):
    """Feng's two-dimensional result, Eq. eq54, with the denominator read as
    3 (1 + R)^2: the printed 3 (1 + 2R)^2 does not reproduce Table 1's Feng column,
    3 (1 + R)^2 does to the printed digits."""
    return Ca / (3.0 * (1.0 + R) ** 2) * (R * R + R + 1.0 - 3.0 * S)


def feng_D_as_printed(R, S, Ca):
    return Ca / (3.0 * (1.0 + 2.0 * R) ** 2) * (R * R + R + 1.0 - 3.0 * S)


# -- hydrodynamics ---------------------------------------------------------------------


def poiseuille(ny, g, nu):
    """Channel flow driven by a body acceleration g between no-slip walls at
    y = -1/2 and ny - 1/2: u(y) = g/(2 nu) (y + 1/2)(ny - 1/2 - y)."""
    y = np.arange(ny, dtype=np.float64)
    return g / (2.0 * nu) * (y + 0.5) * (ny - 0.5 - y)


def cap_contact_angle(phi, wall_row=0, level=0.5):
    """Contact angle (degrees) of a drop sitting on the bottom wall (at y = -1/2),
    from its height h and base width b on the phi = level contour of a circular cap:
    tan(theta/2) = 2h/b."""
    ny, nx = phi.shape
    col = phi[:, :].max(axis=1)
    # height: highest row where the contour is crossed along the drop's centre column
    xc = int(np.argmax(phi.sum(axis=0)))
    c = phi[:, xc]
    j = int(np.where(c >= level)[0].max())
    frac = (c[j] - level) / (c[j] - c[j + 1])
    h = j + frac + 0.5
    # base: width of the phi >= level region on the first row, extrapolated to the wall
    def width_at(row):
        r = phi[row]
        inside = np.where(r >= level)[0]
        a, b = inside.min(), inside.max()
        left = a - (r[a] - level) / (r[a] - r[a - 1])
        right = b + (r[b] - level) / (r[b] - r[b + 1])
        return right - left
    w0 = width_at(0)
    w1 = width_at(1)
    base = w0 + 0.5 * (w0 - w1)
    return math.degrees(2.0 * math.atan(2.0 * h / base))


def cap_contact_line(phi, level=0.5):
    """Contact line of a drop on the bottom wall (at y = -1/2) from a [ny, nx] phi field:
    on rows 0 and 1, the crossings of phi = level interpolated linearly between the
    outermost nodes with phi >= level and their outside neighbours, each extrapolated
    linearly to the wall.  Returns (left, right, radius); NaNs when a row has no such node
    or the span reaches an end of the row."""
    ends = []
    for r in (0, 1):
        row = np.asarray(phi[r], dtype=np.float64)
        inside = np.where(row >= level)[0]
        if inside.size == 0 or inside.min() == 0 or inside.max() == row.size - 1:
            return (math.nan, math.nan, math.nan)
        a, b = int(inside.min()), int(inside.max())
        left = a - (row[a] - level) / (row[a] - row[a - 1])
        right = b + (row[b] - level) / (row[b] - row[b + 1])
        ends.append((left, right))
    left = ends[0][0] + 0.5 * (ends[0][0] - ends[1][0])
    right = ends[0][1] + 0.5 * (ends[0][1] - ends[1][1])
    return (left, right, 0.5 * (right - left))
