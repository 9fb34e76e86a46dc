"""Coupled pins of the oracle's full step (Algorithm 1): the planar-layer problem of
Sec. 6.1 run to its steady state."""
import math

import numpy as np
from scipy import integrate

import analytic as an
from oracle import ehd
from paper_2407_01654_gb300 import workloads as wl


def test_planar_layers_steady_state():
    """Two leaky-dielectric layers between electrodes (permittivity ratio 10, conductivity
    ratio 0.1), run through the full coupled step until the charge has relaxed.  The
    potential matches the diffuse-layer exact profile within 5 % and the sharp-interface
    Eq. weq72 within 15 % (the interface is 4 nodes wide on 32 rows); the interface
    charge obeys Gauss's law Q = J (eps_v/sigma_v - eps_l/sigma_l) within 8 %; the flow
    stays at rest; the potential loop needs one sub-iteration per step once steady."""
    ny = 32
    p, f = wl.planar_layers(nx=4, ny=ny, eps_v=0.5, sigma_v=0.1, alpha=0.002,
                            varphi_high=0.1, width=4.0)
    P = ehd.Params.from_dict(p)
    s = ehd.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    st = s.step(2000)
    F = s.fields()
    yc, W = (ny - 1) / 2, 4.0
    phi_y = lambda t: 0.5 + 0.5 * math.tanh(2 * (yc - t) / W)
    dphi = lambda t: -(1 / W) * (1 - math.tanh(2 * (yc - t) / W) ** 2)
    v_ex, q_ex, E_ex = an.planar_diffuse(
        ny, phi_y, dphi, lambda ph: float(ehd.sigma_of(P, ph)),
        lambda ph: float(ehd.eps_of(P, ph)), lambda ph: float(ehd.deps_dphi(P, ph)),
        lambda ph: P.sigma_l - P.sigma_v, 0.1, 0.0)
    sharp = an.planar_sharp(ny, P.sigma_l / P.sigma_v, 0.1)
    assert an.rel_l2(F["varphi"][:, 0], v_ex) < 0.05
    assert an.rel_l2(F["varphi"][:, 0], sharp) < 0.15
    total, _ = integrate.quad(lambda t: 1 / float(ehd.sigma_of(P, phi_y(t))), -0.5, ny - 0.5,
                              limit=200)
    J = 0.1 / total
    Q = F["q"][:, 0].sum()
    assert abs(Q / (J * (P.eps_v / P.sigma_v - P.eps_l / P.sigma_l)) - 1) < 0.08
    assert np.abs(F["uy"]).max() < 1e-5
    assert st.poisson_iters[-1] == 1
