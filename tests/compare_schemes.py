"""Measurement: the paper's potential LBE against the conventional scheme (Sec. 3.3) on
the GPU -- sub-iterations to the paper's tolerance from a cold start, wall time, and the
accuracy of the potential and field against the exact diffuse-layer solution -- for
planar layers between electrodes at permittivity ratios 10 to 81.

    python tests/compare_schemes.py [--n 128] > table.md
"""
import argparse
import math
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-5)
    args = ap.parse_args()
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    from test_gpu_conventional import layers_gpu
    print(f"planar layers, 4 x {args.n}, walls at potentials 1 and 0, exact steady charge, "
          f"cold start, relative change < {args.tol:g}\n")
    print("| eps ratio | scheme | chi | sub-iterations | GPU s | varphi rel. L2 | E rel. L2 |")
    print("|---|---|---|---|---|---|---|")
    for ratio in (10.0, 20.0, 40.0, 81.0):
        for scheme, chi in ((0, 1.0), (1, 1.0), (1, math.sqrt(ratio)), (1, ratio)):
            t0 = time.perf_counter()
            k, ev, ee = layers_gpu(ehd, args.n, ratio, scheme, chi, args.tol)
            t = time.perf_counter() - t0
            name = "paper (Eq. weq53)" if scheme == 0 else "conventional"
            chis = "-" if scheme == 0 else f"{chi:.3g}"
            print(f"| {ratio:g} | {name} | {chis} | {k} | {t:.2f} | {ev:.3g} | {ee:.3g} |",
                  flush=True)


if __name__ == "__main__":
    main()
