"""The C ABI library builds for sm_103a, loads, exports every entry point declared in
include/ehd.h, and its argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2407_01654_gb300 import build as ehd_build
from paper_2407_01654_gb300 import ehd
from paper_2407_01654_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(ehd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    ehd_build.build()
    return ehd.lib()


def test_every_declared_symbol_exported(L):
    names = declared_functions()
    assert "ehd_create" in names and "ehd_step" in names and "ehd_solve_potential" in names
    for n in names:
        assert hasattr(L, n), n
    # the binding declares exactly the header's functions
    assert set(ehd.SIGNATURES) == set(names)


def test_struct_layouts_match(L):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.ehd_abi_sizes(ctypes.byref(a), ctypes.byref(b)) == 0
    assert a.value == ctypes.sizeof(ehd.Params)
    assert b.value == ctypes.sizeof(ehd.Stats)


def test_strings_and_workspace_size(L):
    assert b"sm_103a" in L.ehd_version()
    assert L.ehd_error_string(0) == b"ok"
    assert L.ehd_error_string(4).startswith(b"potential")
    p = ehd.Params.from_dict(wl.make_params(nx=512, ny=1024))
    nb = ctypes.c_size_t()
    assert L.ehd_workspace_bytes(ctypes.byref(p), ctypes.byref(nb)) == 0
    N = 512 * 1024
    # two copies of 27 + 8 populations, history, fields, staging
    assert nb.value >= 4 * N * (2 * 27 + 2 * 8 + 6 + 1 + 2 + 8 + 1)
    bad = ehd.Params.from_dict(wl.make_params(nx=0, ny=4))
    assert L.ehd_workspace_bytes(ctypes.byref(bad), ctypes.byref(nb)) == 1


@pytest.mark.parametrize("change,code", [
    (dict(nx=0), 1),
    (dict(precision=7), 1),
    (dict(poisson_loop=5), 1),
    (dict(mobility=1e-4), 2),          # tau_g too close to 1/2
    (dict(mu_v=1e-5), 2),              # tau_f too close to 1/2
    (dict(sigma_v=0.9, eps_v=1.0), 2), # sigma/eps above 0.5
    (dict(poisson_min_iter=0), 1),
])
def test_create_rejects_bad_parameters(L, change, code):
    d = wl.make_params(nx=8, ny=8)
    d.update(change)
    p = ehd.Params.from_dict(d)
    h = ctypes.c_void_p()
    assert L.ehd_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == code
    assert not h.value


def workspace(L, **kw):
    p = ehd.Params.from_dict(wl.make_params(**kw))
    nb = ctypes.c_size_t()
    assert L.ehd_workspace_bytes(ctypes.byref(p), ctypes.byref(nb)) == 0
    return nb.value


def test_workspace_holds_the_export_bands_of_each_on_chip_loop(L):
    """Host geometry (no GPU): the workspace reserves, per tile and per copy of the
    double buffer, 8 directions of the export band of the on-chip loop asked for — one,
    two or three nodes wide (2, 4, 6 x (64 + TY) slots).  At 512 x 1024 the tiles are
    8 x 19 of 64 x 56; a narrow, tall 4 x 256 lattice gets 4 tiles of 4 x 64; a lattice
    too large for the chip gets none, whatever the loop."""
    w = {loop: workspace(L, nx=512, ny=1024, poisson_loop=loop) for loop in (2, 3, 4)}
    band = 2 * 152 * 8 * 4  # bytes per band slot over all tiles and both copies
    assert w[3] - w[2] == band * (4 - 2) * (64 + 56)
    assert w[4] - w[3] == band * (6 - 4) * (64 + 56)
    t = {loop: workspace(L, nx=4, ny=256, poisson_loop=loop) for loop in (2, 3)}
    assert t[3] - t[2] == 2 * 4 * 8 * 4 * (4 - 2) * (64 + 64)
    big = {loop: workspace(L, nx=1024, ny=1024, poisson_loop=loop) for loop in (2, 3, 4)}
    assert big[2] == big[3] == big[4]


@pytest.mark.parametrize("nx,ny,ok", [
    (4, 16 * 65536, True),        # 65536 streaming tiles of 64 x 16: the limit
    (4, 16 * 65536 + 1, False),   # one tile row more: N / 256 is far below the limit
    (12, 16 * 65544, False),      # 65544 tiles, while N / 256 = 49158 is within its limit
    (8192, 2048, True),           # 16.8 M nodes, 16384 tiles
])
def test_size_validation_counts_streaming_tiles(L, nx, ny, ok):
    """A lattice is refused (EHD_ERR_INVALID_ARG, from the host-side checks alone) when the
    streaming potential kernel would need more CTAs than the per-CTA partial sums region
    holds, ceil(nx / 64) * ceil(ny / 16) > 65536 -- for narrow, tall lattices that is far
    more than one CTA per 256 nodes."""
    p = ehd.Params.from_dict(wl.make_params(nx=nx, ny=ny))
    nb = ctypes.c_size_t()
    assert L.ehd_workspace_bytes(ctypes.byref(p), ctypes.byref(nb)) == (0 if ok else 1)
    if not ok:
        h = ctypes.c_void_p()
        assert L.ehd_create(ctypes.byref(p), None, 0, None, ctypes.byref(h)) == 1
        assert not h.value


@pytest.mark.parametrize("change,nslabs", [
    (dict(), 0),                    # at least one slab
    (dict(), 65),                   # at most 64
    (dict(ny=3), 4),                # at least one row per slab
    (dict(precision=1), 2),         # FP32 storage only
])
def test_slabs_create_rejects_bad_arguments(L, change, nslabs):
    """The slab decomposition refuses bad arguments on the host, before any device work."""
    d = wl.make_params(nx=16, ny=16)
    d.update(change)
    p = ehd.Params.from_dict(d)
    h = ctypes.c_void_p()
    assert L.ehd_slabs_create(ctypes.byref(p), nslabs, None, ctypes.byref(h)) == 1
    assert not h.value


def test_null_handles_are_refused(L):
    """Entry points given a null simulation handle return EHD_ERR_INVALID_ARG (1) without
    touching the device."""
    out = (ctypes.c_double * 3)()
    assert L.ehd_contact_line(None, ctypes.c_double(0.5), out) == 1
    assert L.ehd_step(None, 1, None) == 1
    assert L.ehd_use_graphs(None, 1) == 1
    assert L.ehd_read_fields(None, 1, None, 0) == 1


def test_grid_exchange_refuses_before_touching_the_device(L):
    """The synchronisation-floor helper checks its arguments first: a null result pointer
    or a lattice with fewer than 3 tiles of 64 x 56 in a direction (its ring would meet the
    same neighbour on both sides) is refused with EHD_ERR_INVALID_ARG (1)."""
    v = ctypes.c_double()
    L.ehd_diag_grid_exchange.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double)]
    assert L.ehd_diag_grid_exchange(None, 512, 1024, None) == 1
    assert L.ehd_diag_grid_exchange(None, 128, 1024, ctypes.byref(v)) == 1  # 2 tiles in x
    assert L.ehd_diag_grid_exchange(None, 512, 112, ctypes.byref(v)) == 1  # 2 tiles in y
    assert L.ehd_diag_grid_exchange(None, 0, 1024, ctypes.byref(v)) == 1


def test_caller_owned_output_buffers_are_checked():
    """read_fields(out=...) passes the caller's arrays to ehd_read_fields only when each has
    the shape and type the call writes (host: C-contiguous float64)."""
    import numpy as np
    good = [np.zeros((6, 4)), np.zeros((6, 4))]
    assert ehd.output_pointers(good, (6, 4), False) == [a.ctypes.data for a in good]
    for bad in (np.zeros((6, 4), np.float32), np.zeros((4, 6)), np.zeros((6, 8))[:, ::2],
                [[0.0] * 4] * 6):
        with pytest.raises(ValueError):
            ehd.output_pointers([bad], (6, 4), False)
    ro = np.zeros((6, 4))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        ehd.output_pointers([ro], (6, 4), False)
    with pytest.raises(ValueError):  # a host array is not a device output
        ehd.output_pointers([np.zeros((6, 4))], (6, 4), True)
