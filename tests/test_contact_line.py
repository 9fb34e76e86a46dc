"""The contact-line extraction behind the contact-radius histories of Sec. 7.2 (Fig. 11),
as the tests' numpy reference (`analytic.cap_contact_line`) computes it, pinned against
circular caps whose contact radius is known in closed form: a cap of radius R centred
hc above the wall (at y = -1/2) meets it at half-width sqrt(R^2 - hc^2)."""
import math

import numpy as np
import pytest

import analytic as an
from paper_2407_01654_gb300 import workloads as wl


def cap(nx, ny, xc, R, hc, width=4.0):
    y, x = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    d = np.sqrt((x - xc) ** 2 + (y - (-0.5 + hc)) ** 2)
    return wl.tanh_profile(R - d, width)


@pytest.mark.parametrize("R,hc", [(20.0, 0.0), (20.0, 8.0), (20.0, -8.0), (30.0, 12.0),
                                  (12.0, 0.0)])
def test_contact_radius_of_circular_caps(R, hc):
    """Radius within 0.05 lattice units of the closed form and centred within 0.02, for
    contact angles below, at and above 90 degrees (hc > 0 is above 90).  Dropping the
    extrapolation to the wall (row 0 alone) is off by 0.2 at hc = +-8, so the pin sees
    it."""
    xc = 63.3
    left, right, radius = an.cap_contact_line(cap(128, 64, xc, R, hc))
    assert abs(radius - math.sqrt(R * R - hc * hc)) < 0.05
    assert abs(0.5 * (left + right) - xc) < 0.02
    if hc != 0.0:
        # row 0's own crossings (row 1 replaced by row 0: no extrapolation)
        flat = cap(128, 64, xc, R, hc)
        flat[1] = flat[0]
        assert abs(an.cap_contact_line(flat)[2] - math.sqrt(R * R - hc * hc)) > 0.1


def test_no_contact_line():
    """No node at or above the level on the wall rows, or a drop across the periodic seam:
    NaN."""
    phi = np.zeros((32, 64))
    assert all(math.isnan(v) for v in an.cap_contact_line(phi))
    seam = cap(64, 32, 0.0, 10.0, 0.0)
    assert all(math.isnan(v) for v in an.cap_contact_line(seam))
