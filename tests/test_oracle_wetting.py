"""Pins of the oracle's wetting boundary rule (Eq. weq68) and the electrowetting
effective angle (Eq. weq69, Sec. 7.2): equilibrium contact angles of sessile drops."""
import math

import numpy as np
import pytest

import analytic as an
from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl


def cap(nx, ny, R, theta_deg, W):
    """Circular cap of radius R meeting the wall y = -1/2 at angle theta."""
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    yc = -0.5 - R * math.cos(math.radians(theta_deg))
    return wl.tanh_profile(R - np.sqrt((x - (nx - 1) / 2) ** 2 + (y - yc) ** 2), W)


def equilibrium_angle(theta_y, ew=0.0, ew_sign=1.0, start=None, steps=1500):
    nx, ny, R = 64, 32, 14
    p = wl.make_params(nx=nx, ny=ny, walls_y=1, gamma=0.03, width=4.0, mobility=0.1,
                       mu_l=0.1, mu_v=0.1, theta_bottom_deg=theta_y, ew_bottom=ew,
                       ew_sign=ew_sign)
    phi0 = cap(nx, ny, R, theta_y if start is None else start, 4.0)
    z = np.zeros((ny, nx))
    s = ehd.Sim(p)
    s.set_fields(phi0, z, z, z)
    s.step(steps)
    return an.cap_contact_angle(s.fields()["phi"])


@pytest.mark.parametrize("theta", [60.0, 90.0, 120.0])
def test_young_angle_kept(theta):
    """A cap at the Young angle stays within 2 degrees of it (Eq. weq68 realises
    cos(theta_Y) of Young's equation, Eq. weq67)."""
    assert abs(equilibrium_angle(theta) - theta) < 2.0


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_electrowetting_angle(sign):
    """Young-Lippmann (Eq. weq69): with eta/d = 0.3 the drop relaxes from 90 degrees to
    cos(theta_B) = cos(theta_Y) + 0.3 (classical) or - 0.3 (reversed, Sec. 7.2), within
    2.5 degrees."""
    target = math.degrees(math.acos(sign * 0.3))
    got = equilibrium_angle(90.0, ew=0.3, ew_sign=sign, start=90.0)
    assert abs(got - target) < 2.5


def test_ramp_and_clamp():
    """The applied wall potential ramps linearly to full value; the electrowetting term
    follows the square of that fraction (eta/d is quadratic in the voltage, Eq. weq69);
    cos(theta_eff) is clamped to [-1, 1]."""
    P = ehd.Params.from_dict(wl.make_params(nx=4, ny=4, varphi_top=2.0, ramp_steps=100,
                                             theta_bottom_deg=90.0, ew_bottom=0.8))
    assert ehd.wall_potentials(P, 0) == (0.0, 0.0)
    assert ehd.wall_potentials(P, 50) == (0.0, 1.0)
    assert ehd.wall_potentials(P, 500) == (0.0, 2.0)
    assert abs(ehd.cos_theta_eff(P, 50)[0] - 0.8 * 0.25) < 1e-15
    P2 = ehd.Params.from_dict(wl.make_params(nx=4, ny=4, theta_bottom_deg=30.0, ew_bottom=0.8))
    assert ehd.cos_theta_eff(P2, 0)[0] == 1.0


def test_each_wall_takes_its_own_young_angle():
    """A cap hanging from the top wall with theta_top = 60 degrees, the bottom wall set to
    120 degrees: it keeps 60 degrees within 2 (the mirror image of the bottom-wall case,
    so each wall's rule reads its own angle)."""
    nx, ny, R = 64, 32, 14
    p = wl.make_params(nx=nx, ny=ny, walls_y=1, gamma=0.03, width=4.0, mobility=0.1,
                       mu_l=0.1, mu_v=0.1, theta_bottom_deg=120.0, theta_top_deg=60.0)
    phi0 = cap(nx, ny, R, 60.0, 4.0)[::-1].copy()
    z = np.zeros((ny, nx))
    s = ehd.Sim(p)
    s.set_fields(phi0, z, z, z)
    s.step(1500)
    assert abs(an.cap_contact_angle(s.fields()["phi"][::-1]) - 60.0) < 2.0
