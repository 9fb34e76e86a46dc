"""The index-checking debug build (libehd_checked.so): on lattices with walls, ramps, partial
tiles and every potential loop, no index the kernels form leaves its field, and the
fields equal the normal build's bit for bit (no index was clamped).  The checked library
runs in a child process, since a process holds one copy of the library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from test_gpu_parity import ALL_FIELDS, droplet_box
from paper_2407_01654_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


CASES = {
    # the sessile drop with its ramped, electrowetting walls on the two-step on-chip loop
    "sessile-132x100-loop3": lambda: wl.sessile_drop(seed=3, nx=132, ny=100, r=30.0,
                                                     ramp_steps=400, start_step=50,
                                                     poisson_loop=3)[:2],
    # a periodic box on the streaming loop and on the one-step loop, FP16 storage too
    "droplet-70x45-loop1": lambda: droplet_box(70, 45, 10.0, seed=4, poisson_loop=1),
    "droplet-70x45-loop2-fp16": lambda: droplet_box(70, 45, 10.0, seed=4, poisson_loop=2,
                                                   precision=1),
}

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
from paper_2407_01654_gb300 import build, ehd
ehd.LIB_PATH = build.build(checked=True)
import test_gpu_checked as t
out = {{}}
for name, make in t.CASES.items():
    p, f = make()
    p["poisson_fixed_iter"] = 7
    g = ehd.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    g.step(12)
    F = g.read_fields()
    out[name] = {{"errors": g.index_errors(),
                 "fields": {{k: np.asarray(v).tobytes().hex() for k, v in F.items()}}}}
    g.close()
assert b"checked" in ehd.lib().ehd_version()
print(json.dumps(out))
"""


def test_checked_build_meets_no_out_of_range_index(gpu):
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for name, make in CASES.items():
        assert got[name]["errors"] == 0, name
        p, f = make()
        p["poisson_fixed_iter"] = 7
        g = gpu.Sim(p)
        g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        g.step(12)
        F = g.read_fields()
        assert g.index_errors() == 0
        g.close()
        for k in ALL_FIELDS:
            assert np.asarray(F[k]).tobytes().hex() == got[name]["fields"][k], (name, k)
