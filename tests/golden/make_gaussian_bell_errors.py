"""Writes gaussian_bell_errors.json: the FP64 oracle's relative L2 error of the charge
against the closed form for the Gaussian-bell charge relaxation of Sec. 6.2 (the
set-up of workloads.gaussian_bell: periodic N x N, s0 = N/16, diffusive scaling), at
N = 64, 128 and 256.  The GPU physics test checks that the CUDA path reaches the same
errors.

Calls only the oracle (and the closed form in tests/analytic.py); nothing here runs the
CUDA library.  Run from the repository root:
    python tests/golden/make_gaussian_bell_errors.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import analytic as an  # noqa: E402
from oracle import ehd as orc  # noqa: E402
from paper_2407_01654_gb300 import workloads as wl  # noqa: E402

SIZES = (64, 128, 256)


def oracle_error(N):
    # with uniform sigma and eps the charge does not depend on the potential
    # (R = -sigma q / eps), so one potential sub-iteration per step suffices
    p, f, n, s0 = wl.gaussian_bell(N, poisson_fixed_iter=1)
    s = orc.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    s.step(n)
    qa = an.gaussian_bell(N, n, s0, f["q"].max(), p["alpha"], p["sigma_v"], p["eps_v"])
    return an.rel_l2(s.fields()["q"], qa), n


def main():
    out = {"source": "FP64 oracle (oracle/ehd.py), Gaussian-bell charge relaxation of "
                     "Sec. 6.2 with diffusion (workloads.gaussian_bell), relative L2 error "
                     "of q against the closed form (tests/analytic.py gaussian_bell) at the "
                     "end time; written by tests/golden/make_gaussian_bell_errors.py",
           "rows": []}
    for N in SIZES:
        t = time.time()
        err, n = oracle_error(N)
        out["rows"].append({"N": N, "steps": n, "rel_l2": err})
        print(f"N={N} steps={n} err={err:.6e} ({time.time() - t:.1f} s)", flush=True)
    with open(os.path.join(HERE, "gaussian_bell_errors.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
