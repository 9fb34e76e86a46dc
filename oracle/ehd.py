"""FP64 CPU oracle of the coupled phase-field lattice Boltzmann (LB) time step for
two-phase electrohydrodynamics (Xiong, Wang, Huang & Luo, arXiv 2407.01654).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg import or run this module.  The library (the CUDA path
behind the C ABI) never imports, links or executes it, and the two share no code:
this file derives every constant and formula from the paper on its own.

What it computes, in the paper's notation and order (Algorithm 1, Sec. 5):

  * D2Q9 lattice (Eq. weq37), c_s^2 = 1/3, lattice units dx = dt = 1.
  * property laws: Hermite permittivity eps(phi), linear rho, mu, sigma (Remark II,
    Eq. weq36); eps_hat = eps - eps_v (Eq. weq52).
  * isotropic FD gradient / Laplacian (Sec. 3.2, the two stencil equations after the
    backward time difference), wall ghost rows from the wetting condition (Eq. weq68)
    with the electrowetting effective angle (Eq. weq69 and Sec. 7.2).
  * hydrodynamic LBE (Eqs. weq38-weq43, eq29, eq32), Cahn-Hilliard LBE (Eqs.
    weq45-weq49), Poisson LBE with the large-ratio discrete forcing (Eqs. weq52-weq55,
    Appendix A Eq. eqA.16), Nernst-Planck LBE (Eqs. weq56-weq62).
  * the Poisson inner loop with the relative-change stopping rule of Algorithm 1.

Every array operation is one term of one equation; there is no fusion, blocking or
reordering beyond what the equations state.  Streaming is written as a pull:
after the step, population i at node x is the post-collision population i of node
x - c_i.  Walls (y direction, half-way between the first/last row and a ghost row):
half-way bounce-back for f, g, l and anti-bounce-back with the wall potential for h.

Readings of passages where the paper is silent or garbled are marked "reading:" at the
place they are used; each is listed with its justification in the design notes.

Parity status of each function: every function here is pinned by a test in
tests/test_oracle_*.py against closed forms, exact moment identities, exact discrete
budgets or the paper's printed values, except where its docstring says
"parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, fields as dc_fields

import numpy as np

# ---------------------------------------------------------------------------------
# Lattice: D2Q9 (Sec. 3, Eq. weq37)
# ---------------------------------------------------------------------------------


def _d2q9_velocities():
    """c_i from the closed formula of Eq. weq37 (c = 1): the rest velocity, four axis
    directions at angles (i-1)pi/2, four diagonals of length sqrt(2) at (2i-9)pi/4."""
    cs = [(0, 0)]
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2
        cs.append((round(math.cos(a)), round(math.sin(a))))
    for i in range(5, 9):
        a = (2 * i - 9) * math.pi / 4
        cs.append((round(math.sqrt(2) * math.cos(a)), round(math.sqrt(2) * math.sin(a))))
    return np.array(cs, dtype=np.int64)


C = _d2q9_velocities()                      # (9, 2) integer lattice velocities
CX = C[:, 0].astype(np.float64)
CY = C[:, 1].astype(np.float64)
# weights (Sec. 3, after Eq. weq37)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
CS2 = 1.0 / 3.0                             # c_s^2 = c^2 / 3
# diffusional weights of the Poisson source (after Eq. weq54)
VARPI = np.array([0.0] + [1 / 8] * 8, dtype=np.float64)
# opposite direction: c_opp(i) = -c_i
OPP = np.array([int(np.where((C == -C[i]).all(axis=1))[0][0]) for i in range(9)])


# ---------------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------------


@dataclass
class Params:
    """Physical and numerical parameters in lattice units.

    Phase "l" is phi = 1, phase "v" is phi = 0 (Sec. 2.2).  x is periodic; y has
    walls (walls_y=True) or is periodic.
    """
    nx: int
    ny: int
    walls_y: bool = True
    rho_l: float = 1.0
    rho_v: float = 1.0
    mu_l: float = 0.1
    mu_v: float = 0.1
    sigma_l: float = 0.0
    sigma_v: float = 0.0
    eps_l: float = 1.0
    eps_v: float = 1.0
    alpha: float = 0.1            # charge diffusivity (Eq. weq56)
    gamma: float = 0.01           # surface tension
    width: float = 4.0            # interface width W
    mobility: float = 0.1         # M
    theta_bottom_deg: float = 90.0
    theta_top_deg: float = 90.0
    ew_bottom: float = 0.0        # electrowetting number eta/d at the bottom wall
    ew_sign: float = 1.0          # +1 classical, -1 reversed electrowetting (Sec. 7.2)
    varphi_bottom: float = 0.0    # Dirichlet potential of the bottom wall
    varphi_top: float = 0.0       # Dirichlet potential of the top wall
    ramp_steps: int = 0           # wall potential ramps linearly from 0 over this many steps
    body_gx: float = 0.0          # optional body acceleration (force rho*g)
    body_gy: float = 0.0
    poisson_tol: float = 1e-5     # Algorithm 1 stopping tolerance
    poisson_max_iter: int = 100000
    poisson_min_iter: int = 1
    poisson_fixed_iter: int = 0   # > 0: exactly this many sub-iterations, no stopping test
    neutralize_charge: bool = False
    start_step: int = 0
    potential_scheme: int = 0     # 0: the paper's scheme (Eq. weq53); 1: conventional
    chi: float = 1.0              # conventional scheme: eps = chi c_s^2 (tau_varphi - 1/2)
    field_mode: int = 0           # E outside the h forcing: 0 local (Eq. eqA.16), 1 stencil
    lagged_field: int = 0         # 1: hbar of step n uses E of step n-1 (Alg. 1's order)

    @classmethod
    def from_dict(cls, d):
        names = {f.name for f in dc_fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})

    # derived coefficients --------------------------------------------------------
    @property
    def beta(self):
        """beta = 12 gamma / W (Sec. 2.2)."""
        return 12.0 * self.gamma / self.width

    @property
    def kappa(self):
        """kappa = 3 gamma W / 2 (Sec. 2.2)."""
        return 3.0 * self.gamma * self.width / 2.0

    @property
    def tau_g(self):
        """M = c_s^2 (tau_g - 1/2) dt (Sec. 3.2)."""
        return 0.5 + self.mobility / CS2

    @property
    def tau_h(self):
        """tau_h = 1/2 + eps_v / (c_s^2 dt) (Sec. 3.3, Eq. eqA.15)."""
        return 0.5 + self.eps_v / CS2

    @property
    def tau_l(self):
        """tau_l = 1/2 + alpha / (c_s^2 dt) (Sec. 3.4, Eq. eqB.15)."""
        return 0.5 + self.alpha / CS2


# ---------------------------------------------------------------------------------
# Property laws (Remark II, Eq. weq36; Eq. weq52)
# ---------------------------------------------------------------------------------


def eps_of(P, phi):
    """Hermite interpolation eps(phi) = eps_v + phi^2 (2 phi - 3)(eps_v - eps_l)."""
    return P.eps_v + phi ** 2 * (2.0 * phi - 3.0) * (P.eps_v - P.eps_l)


def eps_hat_of(P, phi):
    """eps_hat(phi) = phi^2 (2 phi - 3)(eps_v - eps_l) (after Eq. weq52)."""
    return phi ** 2 * (2.0 * phi - 3.0) * (P.eps_v - P.eps_l)


def deps_dphi(P, phi):
    """eps'(phi), the derivative of the Hermite law: 6 phi (phi - 1)(eps_v - eps_l)."""
    return 6.0 * phi * (phi - 1.0) * (P.eps_v - P.eps_l)


def rho_of(P, phi):
    return phi * (P.rho_l - P.rho_v) + P.rho_v


def mu_of(P, phi):
    return phi * (P.mu_l - P.mu_v) + P.mu_v


def sigma_of(P, phi):
    return phi * (P.sigma_l - P.sigma_v) + P.sigma_v


def tau_f_of(P, phi):
    """mu = rho c_s^2 (tau_f - 1/2) (Sec. 3.1), a local relaxation time."""
    return 0.5 + mu_of(P, phi) / (rho_of(P, phi) * CS2)


# ---------------------------------------------------------------------------------
# Boundary helpers
# ---------------------------------------------------------------------------------


def ramp_factor(P, n):
    """Fraction of the wall potential applied at step n.
    reading: linear ramp from 0 over ramp_steps steps, 1 afterwards (no ramp if 0)."""
    if P.ramp_steps <= 0:
        return 1.0
    return min(1.0, n / P.ramp_steps)


def cos_theta_eff(P, n):
    """Effective contact angle cosines (bottom, top) at step n.

    Eq. weq69: cos(theta_B) = cos(theta_Y) + eta/d; Sec. 7.2 flips the sign of the
    electrowetting term for reversed electrowetting.
    reading: the electrowetting number scales with the square of the applied voltage,
    so during a ramp it is (eta/d) * r(n)^2; the result is clamped to [-1, 1].
    """
    r = ramp_factor(P, n)
    cb = math.cos(math.radians(P.theta_bottom_deg)) + P.ew_sign * P.ew_bottom * r * r
    ct = math.cos(math.radians(P.theta_top_deg))
    return max(-1.0, min(1.0, cb)), max(-1.0, min(1.0, ct))


def wall_potentials(P, n):
    r = ramp_factor(P, n)
    return r * P.varphi_bottom, r * P.varphi_top


def extend_with_ghosts(P, theta_field, cos_b, cos_t):
    """Field on an (ny+2, nx+2) frame: x periodic; y walls get ghost rows from the
    wetting condition n_w . grad(phi) = -sqrt(2 beta/kappa) cos(theta) (phi - phi^2)
    (Eq. weq68), n_w the inward wall normal.

    reading: the wall sits half-way between row 0 and ghost row -1, the normal
    derivative is the one-sided difference across it, and (phi - phi^2) is taken at the
    first fluid row: ghost = phi_0 + sqrt(2 beta/kappa) cos(theta) phi_0 (1 - phi_0).
    The top wall is the mirror image.  Diagonal ghost entries use their own column.
    """
    ny, nx = theta_field.shape
    ext = np.empty((ny + 2, nx + 2))
    ext[1:-1, 1:-1] = theta_field
    if P.walls_y:
        a = math.sqrt(2.0 * P.beta / P.kappa)
        b = theta_field[0]
        t = theta_field[-1]
        ext[0, 1:-1] = b + a * cos_b * (b - b * b)
        ext[-1, 1:-1] = t + a * cos_t * (t - t * t)
    else:
        ext[0, 1:-1] = theta_field[-1]
        ext[-1, 1:-1] = theta_field[0]
    ext[:, 0] = ext[:, -2]
    ext[:, -1] = ext[:, 1]
    return ext


def _neighbour(ext, i):
    """Theta(x + c_i) for every node x, read from the ghost frame."""
    ny = ext.shape[0] - 2
    nx = ext.shape[1] - 2
    cx, cy = C[i]
    return ext[1 + cy:1 + cy + ny, 1 + cx:1 + cx + nx]


def gradient(ext):
    """Isotropic gradient (Sec. 3.2): grad Theta = sum_{i != 0} w_i c_i Theta(x + c_i) / c_s^2."""
    gx = np.zeros_like(ext[1:-1, 1:-1])
    gy = np.zeros_like(gx)
    for i in range(1, 9):
        nb = _neighbour(ext, i)
        gx = gx + W[i] * CX[i] * nb / CS2
        gy = gy + W[i] * CY[i] * nb / CS2
    return gx, gy


def laplacian(ext):
    """Isotropic Laplacian (Sec. 3.2): sum_{i != 0} 2 w_i [Theta(x + c_i) - Theta(x)] / c_s^2."""
    centre = ext[1:-1, 1:-1]
    lap = np.zeros_like(centre)
    for i in range(1, 9):
        lap = lap + 2.0 * W[i] * (_neighbour(ext, i) - centre) / CS2
    return lap


def stream(P, post, kind, varphi_w=(0.0, 0.0)):
    """Streaming step f_i(x + c_i, t + 1) = f_i*(x, t), written as a pull.

    kind "bb": half-way bounce-back at the y walls: a population that would enter from
    outside is the post-collision population of the opposite direction at the same
    node (Sec. 6.1 / Sec. 7.1 use half-way bounce-back for the walls).
    kind "abb": anti-bounce-back with a Dirichlet value for the potential LBE:
    h_i = -h*_opp(i) + 2 w_i varphi_w.
    reading: the paper fixes the wall potentials but not how h realises them; the
    anti-bounce-back is the standard second-order Dirichlet rule for an equilibrium of
    the form w_i varphi.
    """
    new = np.empty_like(post)
    ny = post.shape[1]
    for i in range(9):
        cx, cy = C[i]
        s = np.roll(post[i], shift=(cy, cx), axis=(0, 1))
        if P.walls_y and cy != 0:
            row = 0 if cy == 1 else ny - 1
            wall = 0 if cy == 1 else 1
            if kind == "bb":
                s[row, :] = post[OPP[i]][row, :]
            else:
                s[row, :] = -post[OPP[i]][row, :] + 2.0 * W[i] * varphi_w[wall]
        new[i] = s
    return new


# ---------------------------------------------------------------------------------
# Equilibria and discrete source terms
# ---------------------------------------------------------------------------------


def s_i(ux, uy):
    """s_i(u) = w_i [c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)] (Eq. eq29)."""
    out = np.empty((9,) + np.shape(ux))
    uu = ux * ux + uy * uy
    for i in range(9):
        cu = CX[i] * ux + CY[i] * uy
        out[i] = W[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2))
    return out


def f_eq(P, p, rho, ux, uy):
    """Eq. weq40: f_0 = (w_0 - 1) p / c_s^2 + rho s_0, f_i = w_i p / c_s^2 + rho s_i."""
    s = s_i(ux, uy)
    out = np.empty_like(s)
    out[0] = (W[0] - 1.0) * p / CS2 + rho * s[0]
    for i in range(1, 9):
        out[i] = W[i] * p / CS2 + rho * s[i]
    return out


def f_force(P, ux, uy, grho_x, grho_y, Fx, Fy):
    """R_bar_i = w_i [u.grad(rho) + c_i.F/c_s^2 + u grad(rho):(c_i c_i - c_s^2 I)/c_s^2]
    (Eq. weq39); u grad(rho):(c_i c_i - c_s^2 I) = (c_i.u)(c_i.grad rho) - c_s^2 u.grad rho."""
    out = np.empty((9,) + np.shape(ux))
    ug = ux * grho_x + uy * grho_y
    for i in range(9):
        cF = CX[i] * Fx + CY[i] * Fy
        tensor = (CX[i] * ux + CY[i] * uy) * (CX[i] * grho_x + CY[i] * grho_y) - CS2 * ug
        out[i] = W[i] * (ug + cF / CS2 + tensor / CS2)
    return out


def g_eq(P, phi, mu_c):
    """Eq. weq46: g_0 = phi - (1 - w_0) hbar, g_i = w_i hbar."""
    out = np.empty((9,) + phi.shape)
    out[0] = phi - (1.0 - W[0]) * mu_c
    for i in range(1, 9):
        out[i] = W[i] * mu_c
    return out


def g_source(s_adv):
    """G_i = w_i (u.grad phi) [-1 + I:(c_i c_i - c_s^2 I)/(2 c_s^2)] (Eq. weq47).
    In two dimensions I:(c_i c_i - c_s^2 I) = |c_i|^2 - 2 c_s^2."""
    out = np.empty((9,) + np.shape(s_adv))
    for i in range(9):
        trace = CX[i] ** 2 + CY[i] ** 2 - 2.0 * CS2
        out[i] = W[i] * s_adv * (-1.0 + trace / (2.0 * CS2))
    return out


def h_eq(varphi):
    """Eq. weq54: h_0 = (w_0 - 1) varphi, h_i = w_i varphi."""
    out = np.empty((9,) + varphi.shape)
    out[0] = (W[0] - 1.0) * varphi
    for i in range(1, 9):
        out[i] = W[i] * varphi
    return out


def l_eq(q, ux, uy):
    """Eq. weq61: l_i = w_i q (1 + c_i.u / c_s^2)."""
    out = np.empty((9,) + q.shape)
    for i in range(9):
        out[i] = W[i] * q * (1.0 + (CX[i] * ux + CY[i] * uy) / CS2)
    return out


# ---------------------------------------------------------------------------------
# Chemical potential, body force, charge source (Eqs. weq30, weq31, weq57)
# ---------------------------------------------------------------------------------


def chemical_potential(P, phi, lap_phi, Ex, Ey):
    """hbar = 4 beta phi (phi - 1/2)(phi - 1) - kappa lap(phi) - eps'(phi) |E|^2 / 2
    (Eq. weq31)."""
    return (4.0 * P.beta * phi * (phi - 0.5) * (phi - 1.0) - P.kappa * lap_phi
            - 0.5 * deps_dphi(P, phi) * (Ex * Ex + Ey * Ey))


def body_force(P, mu_c, gphi_x, gphi_y, q, Ex, Ey, rho):
    """F = hbar grad(phi) + q E (Eq. weq30; the -grad(alpha q^2/sigma)/2 part of Eq. weq26
    is carried by the modified pressure) plus an optional body force rho g (the paper
    neglects gravity, Sec. 2.1)."""
    return (mu_c * gphi_x + q * Ex + rho * P.body_gx,
            mu_c * gphi_y + q * Ey + rho * P.body_gy)


def charge_source(P, phi, q, gphi_x, gphi_y, Ex, Ey):
    """R = -sigma q / eps + (sigma/eps) grad(eps).E - grad(sigma).E (Eq. weq57).
    reading: grad eps = eps'(phi) grad phi and grad sigma = (sigma_l - sigma_v) grad phi,
    with grad phi from the isotropic stencil (only phi needs a stencil)."""
    eps = eps_of(P, phi)
    sig = sigma_of(P, phi)
    geps_x = deps_dphi(P, phi) * gphi_x
    geps_y = deps_dphi(P, phi) * gphi_y
    gsig_x = (P.sigma_l - P.sigma_v) * gphi_x
    gsig_y = (P.sigma_l - P.sigma_v) * gphi_y
    return (-sig * q / eps + (sig / eps) * (geps_x * Ex + geps_y * Ey)
            - (gsig_x * Ex + gsig_y * Ey))


# ---------------------------------------------------------------------------------
# Potential LBE moments (Eq. weq55, Eq. eqA.16)
# ---------------------------------------------------------------------------------


def varphi_of(h):
    """varphi = sum_{i != 0} h_i / (1 - w_0) (Eq. weq55)."""
    return h[1:].sum(axis=0) / (1.0 - W[0])


def grad_varphi_local(P, h, eps_hat):
    """Local potential gradient (Eq. eqA.16):
    grad varphi = - sum_i c_i h_i / (eps_hat + c_s^2 tau_h dt)."""
    mx = sum(CX[i] * h[i] for i in range(9))
    my = sum(CY[i] * h[i] for i in range(9))
    den = eps_hat + CS2 * P.tau_h
    return -mx / den, -my / den


def poisson_collide(P, h, eps_hat, qsrc):
    """One collision of the potential LBE (Eq. weq53):
    h* = h - (h - h_eq)/tau_h - (eps_hat/c_s^2) w_i c_i.grad(varphi)/tau_h + dt varpi_i q.

    reading: grad(varphi) in the forcing is the potential gradient of Eq. eqA.16
    (Algorithm 1 prints "grad phi^n", taken as a typo for the potential), evaluated from
    the same pre-collision h.
    """
    varphi = varphi_of(h)
    gx, gy = grad_varphi_local(P, h, eps_hat)
    heq = h_eq(varphi)
    out = np.empty_like(h)
    for i in range(9):
        forcing = (eps_hat / CS2) * W[i] * (CX[i] * gx + CY[i] * gy) / P.tau_h
        out[i] = h[i] - (h[i] - heq[i]) / P.tau_h - forcing + VARPI[i] * qsrc
    return out


# The conventional potential LBE (Sec. 3.3, the scheme of Chai et al. the paper compares
# against): no discrete forcing; instead the relaxation time follows the permittivity,
# eps(phi) = chi c_s^2 (tau_varphi - 1/2) dt with an artificial factor chi.


def tau_phi_conventional(P, phi):
    """tau_varphi(x) = 1/2 + eps(phi(x)) / (chi c_s^2 dt), from the relation of Sec. 3.3."""
    return 0.5 + eps_of(P, phi) / (P.chi * CS2)


def grad_varphi_conventional(P, h, tau_phi):
    """Local potential gradient of the conventional scheme: its first moment relaxes with
    tau_varphi, sum_i c_i h_i = -c_s^2 tau_varphi dt grad varphi (Eq. eqA.16 with
    eps_hat = 0 and tau_h replaced by the local tau_varphi)."""
    mx = sum(CX[i] * h[i] for i in range(9))
    my = sum(CY[i] * h[i] for i in range(9))
    den = CS2 * tau_phi
    return -mx / den, -my / den


def poisson_collide_conventional(P, h, tau_phi, qsrc):
    """One collision of the conventional potential LBE:
    h* = h - (h - h_eq)/tau_varphi + dt varpi_i q / chi.
    Its steady state solves div(c_s^2 (tau_varphi - 1/2) grad varphi) + q / chi = 0, which
    is div(eps grad varphi) + q = 0 (the equation before Eq. weq52) divided by chi."""
    heq = h_eq(varphi_of(h))
    out = np.empty_like(h)
    for i in range(9):
        out[i] = h[i] - (h[i] - heq[i]) / tau_phi + VARPI[i] * qsrc / P.chi
    return out


def potential_gradient(P, h, phi):
    """grad varphi from the local first moment of the scheme in use (phi: the phase field
    the potential was solved with)."""
    if P.potential_scheme == 1:
        return grad_varphi_conventional(P, h, tau_phi_conventional(P, phi))
    return grad_varphi_local(P, h, eps_hat_of(P, phi))


def extend_potential_with_ghosts(P, varphi, varphi_w):
    """varphi on an (ny+2, nx+2) frame for the stencil: x periodic; at a wall half-way
    between row 0 and the ghost row the potential is the Dirichlet value varphi_w, so the
    ghost row is its linear extension 2 varphi_w - varphi(row 0) (top wall alike).
    reading: the paper gives no stencil rule for varphi at an electrode."""
    ny, nx = varphi.shape
    ext = np.empty((ny + 2, nx + 2))
    ext[1:-1, 1:-1] = varphi
    if P.walls_y:
        ext[0, 1:-1] = 2.0 * varphi_w[0] - varphi[0]
        ext[-1, 1:-1] = 2.0 * varphi_w[1] - varphi[-1]
    else:
        ext[0, 1:-1] = varphi[-1]
        ext[-1, 1:-1] = varphi[0]
    ext[:, 0] = ext[:, -2]
    ext[:, -1] = ext[:, 1]
    return ext


def electric_field(P, h, phi, varphi_w):
    """E = -grad varphi for the chemical potential, force and charge source (a4).
    field_mode 0: the local first moment of the scheme in use (Eq. eqA.16); field_mode 1:
    the isotropic stencil of Sec. 3.2 on varphi of Eq. weq55 (the variant of the reading
    that E outside the h forcing is local)."""
    if P.field_mode == 1:
        gx, gy = gradient(extend_potential_with_ghosts(P, varphi_of(h), varphi_w))
    else:
        gx, gy = potential_gradient(P, h, phi)
    return -gx, -gy


def poisson_solve(P, h, phi, q, varphi_w, tol=None, max_iter=None, fixed_iter=None,
                  min_iter=None):
    """Poisson inner loop of Algorithm 1 (step 3) with phi and q held fixed.

    Each sub-iteration is a collision (Eq. weq53) and a stream; the loop stops once
    sqrt(sum (varphi^{k+1} - varphi^k)^2 / sum (varphi^k)^2) < tol (Algorithm 1).
    reading: at least min_iter sub-iterations are made; 0/0 counts as converged;
    max_iter caps the loop (not converged).  fixed_iter > 0 runs exactly that many
    sub-iterations with no stopping test.
    Returns (h, iterations, last relative change, converged).
    """
    tol = P.poisson_tol if tol is None else tol
    max_iter = P.poisson_max_iter if max_iter is None else max_iter
    fixed_iter = P.poisson_fixed_iter if fixed_iter is None else fixed_iter
    min_iter = P.poisson_min_iter if min_iter is None else min_iter
    eps_hat = eps_hat_of(P, phi)
    tau_phi = tau_phi_conventional(P, phi) if P.potential_scheme == 1 else None
    qsrc = q - q.mean() if P.neutralize_charge else q
    varphi_old = varphi_of(h)
    it = 0
    rel = math.inf
    while True:
        if P.potential_scheme == 1:
            post = poisson_collide_conventional(P, h, tau_phi, qsrc)
        else:
            post = poisson_collide(P, h, eps_hat, qsrc)
        h = stream(P, post, "abb", varphi_w)
        it += 1
        varphi_new = varphi_of(h)
        num = float(np.sum((varphi_new - varphi_old) ** 2))
        den = float(np.sum(varphi_old ** 2))
        if num == 0.0 and den == 0.0:
            rel = 0.0
        elif den == 0.0:
            rel = math.inf
        else:
            rel = math.sqrt(num / den)
        varphi_old = varphi_new
        if fixed_iter > 0:
            if it >= fixed_iter:
                return h, it, rel, True
            continue
        if it >= min_iter and rel < tol:
            return h, it, rel, True
        if it >= max_iter:
            return h, it, rel, False


# ---------------------------------------------------------------------------------
# The coupled simulation
# ---------------------------------------------------------------------------------


FIELD_NAMES = ("phi", "q", "varphi", "Ex", "Ey", "ux", "uy", "p", "mu")


@dataclass
class StepStats:
    steps: int = 0
    poisson_iters: list = field(default_factory=list)
    last_rel_change: float = 0.0
    sum_phi: float = 0.0
    sum_q: float = 0.0
    all_converged: bool = True


class Sim:
    """State of one simulation: post-stream g, l, f at level n, the warm potential
    distribution h, and the history of the lagged quantities
    (R^{n-1}, F^{n-1} for the moment closures, (u.grad phi)^{n-1} and (q u)^{n-1} for the
    backward time differences)."""

    def __init__(self, params):
        self.P = params if isinstance(params, Params) else Params.from_dict(params)
        P = self.P
        shape = (P.ny, P.nx)
        self.n = P.start_step
        self.g = np.zeros((9,) + shape)
        self.l = np.zeros((9,) + shape)
        self.f = np.zeros((9,) + shape)
        self.h = np.zeros((9,) + shape)
        self.R_prev = np.zeros(shape)
        self.Fx_prev = np.zeros(shape)
        self.Fy_prev = np.zeros(shape)
        self.s_prev = np.zeros(shape)
        self.Jx_prev = np.zeros(shape)
        self.Jy_prev = np.zeros(shape)
        self.history_valid = False
        self.phi_poisson = np.zeros(shape)   # phi the last Poisson solve used
        self.vw_poisson = (0.0, 0.0)         # wall potentials of the last Poisson solve
        self.Ex_prev = np.zeros(shape)       # E of the previous step (lagged_field)
        self.Ey_prev = np.zeros(shape)

    # -- initialisation (Algorithm 1, step 1) ---------------------------------------
    def set_fields(self, phi0, q0, ux0, uy0, p0=None):
        """Populations at equilibrium with the given fields, then a potential solve.

        reading: g = g_eq(phi0, hbar(phi0, E = 0)), l = l_eq(q0, u0),
        f = f_eq(p0 (default 0), u0); h starts at h_eq of the potential interpolated
        linearly between the walls (0 if y is periodic) and is then solved to the
        tolerance; the lagged R and F are 0 so that q^0 = q0 and u^0 = u0, and the
        backward time differences are 0 at the first step.
        """
        P = self.P
        phi0 = np.asarray(phi0, dtype=np.float64)
        q0 = np.asarray(q0, dtype=np.float64)
        ux0 = np.asarray(ux0, dtype=np.float64)
        uy0 = np.asarray(uy0, dtype=np.float64)
        p0 = np.zeros_like(phi0) if p0 is None else np.asarray(p0, dtype=np.float64)
        cb, ct = cos_theta_eff(P, self.n)
        ext = extend_with_ghosts(P, phi0, cb, ct)
        lap = laplacian(ext)
        mu_c = 4.0 * P.beta * phi0 * (phi0 - 0.5) * (phi0 - 1.0) - P.kappa * lap
        self.g = g_eq(P, phi0, mu_c)
        self.l = l_eq(q0, ux0, uy0)
        self.f = f_eq(P, p0, rho_of(P, phi0), ux0, uy0)
        vb, vt = wall_potentials(P, self.n)
        if P.walls_y:
            # wall at y = -1/2 and y = ny - 1/2
            y = np.arange(P.ny, dtype=np.float64)
            frac = (y + 0.5) / P.ny
            lin = vb + (vt - vb) * frac
            varphi_lin = np.repeat(lin[:, None], P.nx, axis=1)
        else:
            varphi_lin = np.zeros((P.ny, P.nx))
        self.h = h_eq(varphi_lin)
        self.R_prev[:] = 0.0
        self.Fx_prev[:] = 0.0
        self.Fy_prev[:] = 0.0
        self.s_prev[:] = 0.0
        self.Jx_prev[:] = 0.0
        self.Jy_prev[:] = 0.0
        self.history_valid = False
        return self.solve_potential()

    # -- moments (a1) ----------------------------------------------------------------
    def _moments(self):
        """phi = sum g (Eq. weq49); q = sum l + R^{n-1}/2 (Algorithm 1 step 4, Eq. weq62);
        rho u = sum c f + F^{n-1}/2 (Algorithm 1 step 5, Eq. weq43)."""
        P = self.P
        phi = self.g.sum(axis=0)
        q = self.l.sum(axis=0) + 0.5 * self.R_prev
        rho = rho_of(P, phi)
        ux = (sum(CX[i] * self.f[i] for i in range(9)) + 0.5 * self.Fx_prev) / rho
        uy = (sum(CY[i] * self.f[i] for i in range(9)) + 0.5 * self.Fy_prev) / rho
        return phi, q, rho, ux, uy

    def _pressure(self, phi, rho, ux, uy, gphi_x, gphi_y):
        """p = c_s^2/(1 - w_0) [sum_{i != 0} f_i + (dt/2) u.grad rho + rho s_0(u)] (Eq. eq32),
        grad rho = (rho_l - rho_v) grad phi (rho linear in phi)."""
        P = self.P
        grho_x = (P.rho_l - P.rho_v) * gphi_x
        grho_y = (P.rho_l - P.rho_v) * gphi_y
        s0 = s_i(ux, uy)[0]
        return CS2 / (1.0 - W[0]) * (self.f[1:].sum(axis=0)
                                       + 0.5 * (ux * grho_x + uy * grho_y) + rho * s0)

    def solve_potential(self, tol=None, max_iter=None):
        """The Poisson inner loop alone, for the phi and q of the current populations."""
        phi, q, _, _, _ = self._moments()
        vw = wall_potentials(self.P, self.n)
        self.h, it, rel, ok = poisson_solve(self.P, self.h, phi, q, vw, tol=tol,
                                            max_iter=max_iter)
        self.phi_poisson = phi
        self.vw_poisson = vw
        return it, rel, ok

    # -- one coupled step (Algorithm 1, steps 2-6) -------------------------------------
    def step(self, nsteps=1):
        """Advance nsteps time steps.

        reading (order within a step): all three single-pass LBEs collide with level-n
        fields, as Algorithm 1 writes them (g^{eq,n}, eps_hat^n, q^n, S^n, R^n, F^n); the
        potential loop runs first on (phi^n, q^n) so that hbar^n, F^n and R^n use the
        field E^n of that loop.  E everywhere is the local gradient of Eq. eqA.16.
        """
        stats = StepStats()
        for _ in range(nsteps):
            it, rel, ok = self._one_step()
            if not np.isfinite(self.g[0]).all():
                raise FloatingPointError(f"non-finite populations after step {self.n}")
            stats.steps += 1
            stats.poisson_iters.append(it)
            stats.last_rel_change = rel
            stats.all_converged = stats.all_converged and ok
        phi, q, _, _, _ = self._moments()
        stats.sum_phi = float(phi.sum())
        stats.sum_q = float(q.sum())
        return stats

    def _one_step(self):
        P = self.P
        n = self.n
        # a1: moments and properties at level n
        phi, q, rho, ux, uy = self._moments()
        # a2: stencils on phi with the wetting ghost rows
        cb, ct = cos_theta_eff(P, n)
        ext = extend_with_ghosts(P, phi, cb, ct)
        gphi_x, gphi_y = gradient(ext)
        lap_phi = laplacian(ext)
        # a3: Poisson sub-iterations on (phi^n, q^n)
        vw = wall_potentials(P, n)
        self.h, it, rel, ok = poisson_solve(P, self.h, phi, q, vw)
        self.phi_poisson = phi
        self.vw_poisson = vw
        # a4: E = -grad varphi from the converged h (Eq. eqA.16, or the stencil variant)
        Ex, Ey = electric_field(P, self.h, phi, vw)
        # a5: chemical potential (Eq. weq31), force (Eq. weq30), charge source (Eq. weq57).
        # lagged_field: Algorithm 1 lists the Cahn-Hilliard LBE before the potential solve,
        # so hbar there can only see the previous step's field (the same at the first step)
        if P.lagged_field and self.history_valid:
            mu_c = chemical_potential(P, phi, lap_phi, self.Ex_prev, self.Ey_prev)
        else:
            mu_c = chemical_potential(P, phi, lap_phi, Ex, Ey)
        Fx, Fy = body_force(P, mu_c, gphi_x, gphi_y, q, Ex, Ey, rho)
        R = charge_source(P, phi, q, gphi_x, gphi_y, Ex, Ey)
        p = self._pressure(phi, rho, ux, uy, gphi_x, gphi_y)
        # history at the first step: backward differences vanish
        s_adv = ux * gphi_x + uy * gphi_y
        Jx = q * ux
        Jy = q * uy
        if not self.history_valid:
            s_prev, Jx_prev, Jy_prev = s_adv, Jx, Jy
        else:
            s_prev, Jx_prev, Jy_prev = self.s_prev, self.Jx_prev, self.Jy_prev
        # a6: Cahn-Hilliard LBE (Eq. weq45) with dt G + dt^2/2 d_t G, d_t G backward
        geq = g_eq(P, phi, mu_c)
        G = g_source(s_adv)
        G_prev = g_source(s_prev)
        g_post = self.g - (self.g - geq) / P.tau_g + G + 0.5 * (G - G_prev)
        # a7: Nernst-Planck LBE (Eqs. weq58-weq61)
        leq = l_eq(q, ux, uy)
        pref = 1.0 - 1.0 / (2.0 * P.tau_l)
        l_post = np.empty_like(self.l)
        for i in range(9):
            S_i = pref * W[i] * R
            T_i = pref * W[i] * (CX[i] * (Jx - Jx_prev) + CY[i] * (Jy - Jy_prev)) / CS2
            l_post[i] = self.l[i] - (self.l[i] - leq[i]) / P.tau_l + S_i + T_i
        # a8: hydrodynamic LBE (Eqs. weq38-weq40)
        tau_f = tau_f_of(P, phi)
        feq = f_eq(P, p, rho, ux, uy)
        grho_x = (P.rho_l - P.rho_v) * gphi_x
        grho_y = (P.rho_l - P.rho_v) * gphi_y
        Rbar = f_force(P, ux, uy, grho_x, grho_y, Fx, Fy)
        f_post = self.f - (self.f - feq) / tau_f + (1.0 - 1.0 / (2.0 * tau_f)) * Rbar
        # streaming with half-way bounce-back
        self.g = stream(P, g_post, "bb")
        self.l = stream(P, l_post, "bb")
        self.f = stream(P, f_post, "bb")
        # a9: history for step n+1
        self.R_prev = R
        self.Fx_prev = Fx
        self.Fy_prev = Fy
        self.s_prev = s_adv
        self.Jx_prev = Jx
        self.Jy_prev = Jy
        self.Ex_prev = Ex
        self.Ey_prev = Ey
        self.history_valid = True
        self.n += 1
        return it, rel, ok

    # -- observation -------------------------------------------------------------------
    def fields(self):
        """Macroscopic fields of the current state.

        phi, q, ux, uy, p are those of the current populations (level n); varphi, Ex,
        Ey are those of the last potential solve, which used phi^{n-1}, q^{n-1} after a
        step (Algorithm 1 solves the potential at the start of each step).
        reading: mu, the chemical potential hbar of Eq. weq31 for output, takes the
        current phi (its Laplacian with the current wall rule) and the field Ex, Ey
        returned here (the last solve's); at a steady state the two levels coincide.
        """
        P = self.P
        phi, q, rho, ux, uy = self._moments()
        cb, ct = cos_theta_eff(P, self.n)
        ext = extend_with_ghosts(P, phi, cb, ct)
        gx, gy = gradient(ext)
        p = self._pressure(phi, rho, ux, uy, gx, gy)
        varphi = varphi_of(self.h)
        Ex, Ey = electric_field(P, self.h, self.phi_poisson, self.vw_poisson)
        mu = chemical_potential(P, phi, laplacian(ext), Ex, Ey)
        return {"phi": phi, "q": q, "varphi": varphi, "Ex": Ex, "Ey": Ey,
                "ux": ux, "uy": uy, "p": p, "mu": mu}
