"""Measurement: sensitivity of the droplet deformation (Sec. 7.1, Table 1 rows; 256^2,
r = 40, 30 000 steps) to the two readings of the field outside the potential forcing --
local first moment or stencil on varphi, this step's or the previous step's field in hbar.

    python tests/field_modes_table1.py     (GPU; prints a markdown table)
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import analytic as an  # noqa: E402
from paper_2407_01654_gb300 import workloads as wl  # noqa: E402
from test_gpu_physics import deformation  # noqa: E402

ROWS = [(5.0, 5.0, 0.2, 0.03503), (1.0, 2.0, 0.2, -0.04102), (1.75, 3.5, 0.1, -0.01968),
        (4.75, 3.5, 0.1, 0.02236)]
MODES = [("local, E^n", {}), ("stencil, E^n", {"field_mode": 1}),
         ("local, E^{n-1} in hbar", {"lagged_field": 1}),
         ("stencil, E^{n-1} in hbar", {"field_mode": 1, "lagged_field": 1})]


def run(ehd, R, S, Ca, mode, steps=30000):
    p, f, _ = wl.droplet(N=256, R=R, S=S, Ca=Ca, **mode)
    g = ehd.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    g.step(steps)
    D = deformation(g.read_fields(("phi",))["phi"])
    g.close()
    return D


def main():
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    head = " | ".join(m[0] for m in MODES)
    print(f"| R | S | Ca_E | paper | Feng (2-D) | {head} |")
    print("|---" * (5 + len(MODES)) + "|")
    for R, S, Ca, present in ROWS:
        ds = [run(ehd, R, S, Ca, m[1]) for m in MODES]
        cells = " | ".join(f"{d:.5f}" for d in ds)
        print(f"| {R:g} | {S:g} | {Ca:g} | {present:.5f} | {an.feng_D(R, S, Ca):.5f} | {cells} |",
              flush=True)


if __name__ == "__main__":
    main()
