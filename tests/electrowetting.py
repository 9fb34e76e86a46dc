"""Electrowetting equilibrium (Sec. 6.3, Fig. 4): a conductive drop (r = 25) on the bottom
electrode of a 200 x 100 box, density and viscosity ratio 100, permittivity ratio 81,
W = 4.  Stage 1 relaxes the drop to its Young angle without a field; stage 2 applies
the wall potentials and the electrowetting number eta/d of the wetting rule (Eq. weq69)
and relaxes again.  The apparent angle's cosine should follow Young-Lippmann,
cos(theta_B) = cos(theta_Y) + eta/d.

    python tests/electrowetting.py     (GPU; prints a markdown table)
"""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import analytic as an  # noqa: E402
from paper_2407_01654_gb300 import workloads as wl  # noqa: E402

NX, NY, R, W = 200, 100, 25.0, 4.0
EW = (0.0, 0.1, 0.2, 0.3, 0.4, 0.5)


def params(theta, ew, voltage, eps_v):
    """Drop (phase l) conductive, surrounding gas insulating; bottom electrode at the high
    potential, top wall at 0; no ramp."""
    return wl.make_params(
        nx=NX, ny=NY, walls_y=1, rho_l=1.0, rho_v=0.01, mu_l=0.1, mu_v=0.001, eps_v=eps_v,
        eps_l=81.0 * eps_v, sigma_l=0.05, sigma_v=0.0, alpha=0.01, gamma=0.01, width=W,
        mobility=0.05, theta_bottom_deg=theta, theta_top_deg=90.0, ew_bottom=ew, ew_sign=1.0,
        varphi_bottom=voltage, varphi_top=0.0)


def sweep(ehd, theta_y=110.0, voltage=0.1, eps_v=1.0, steps1=20000, steps2=20000, ew=EW):
    """Returns (theta after stage 1, [(eta/d, theta_B)])."""
    y, x = np.meshgrid(np.arange(NY, dtype=float), np.arange(NX, dtype=float), indexing="ij")
    phi0 = wl.tanh_profile(R - np.sqrt((x - (NX - 1) / 2) ** 2 + (y + 0.5) ** 2), W)
    z = np.zeros((NY, NX))
    s = ehd.Sim(params(theta_y, 0.0, 0.0, eps_v))
    s.set_fields(phi0, z, z, z)
    s.step(steps1)
    F = s.read_fields(("phi", "q", "ux", "uy"))
    s.close()
    theta1 = an.cap_contact_angle(F["phi"])
    out = []
    for e in ew:
        s2 = ehd.Sim(params(theta_y, e, voltage, eps_v))
        s2.set_fields(F["phi"], F["q"], F["ux"], F["uy"])
        st = s2.step(steps2)
        if st["status"] != 0:
            raise RuntimeError(f"stage 2 failed with status {st['status']}")
        out.append((e, an.cap_contact_angle(s2.read_fields(("phi",))["phi"])))
        s2.close()
    return theta1, out


def main():
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    print("| theta_Y | eps_v (eps_l = 81 eps_v) | eta/d | theta_B | cos theta_B | "
          "Young-Lippmann |")
    print("|---|---|---|---|---|---|")
    for eps_v in (1.0, 0.5):
        theta1, pts = sweep(ehd, eps_v=eps_v)
        for e, th in pts:
            cb = math.cos(math.radians(th))
            yl = math.cos(math.radians(110.0)) + e
            print(f"| 110 | {eps_v:g} | {e:g} | {th:.2f} | {cb:.4f} | {yl:.4f} |", flush=True)
        e = np.array([p[0] for p in pts])
        c = np.array([math.cos(math.radians(p[1])) for p in pts])
        slope, icpt = np.polyfit(e, c, 1)
        print(f"| fit | {eps_v:g} | slope {slope:.4f} | intercept {icpt:.4f} | "
              f"stage-1 angle {theta1:.2f} | |", flush=True)


if __name__ == "__main__":
    main()
