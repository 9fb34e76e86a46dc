"""Thin ctypes binding of the CUDA library libehd.so (C ABI in include/ehd.h).

Argument marshalling only: every step of the method runs in the library's kernels.
PyTorch, when used, only provides device memory (the workspace, device field buffers)
and the CUDA stream.  There is no CPU fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libehd.so")

EHD_OK = 0
STATUS = {0: "EHD_OK", 1: "EHD_ERR_INVALID_ARG", 2: "EHD_ERR_UNSTABLE_PARAMS",
          3: "EHD_ERR_NOMEM", 4: "EHD_ERR_NOT_CONVERGED", 5: "EHD_ERR_NONFINITE",
          6: "EHD_ERR_BUSY", 7: "EHD_ERR_CUDA", 8: "EHD_ERR_TOO_LARGE", 9: "EHD_ERR_TIMEOUT"}
EHD_HOST, EHD_DEVICE = 0, 1
FIELDS = ("phi", "q", "varphi", "Ex", "Ey", "ux", "uy", "p", "mu")


class EhdError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("walls_y", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double),
        ("mu_l", ctypes.c_double), ("mu_v", ctypes.c_double),
        ("sigma_l", ctypes.c_double), ("sigma_v", ctypes.c_double),
        ("eps_l", ctypes.c_double), ("eps_v", ctypes.c_double), ("alpha", ctypes.c_double),
        ("gamma", ctypes.c_double), ("width", ctypes.c_double), ("mobility", ctypes.c_double),
        ("theta_bottom_deg", ctypes.c_double), ("theta_top_deg", ctypes.c_double),
        ("ew_bottom", ctypes.c_double), ("ew_sign", ctypes.c_double),
        ("varphi_bottom", ctypes.c_double), ("varphi_top", ctypes.c_double),
        ("ramp_steps", ctypes.c_int32), ("neutralize_charge", ctypes.c_int32),
        ("body_gx", ctypes.c_double), ("body_gy", ctypes.c_double),
        ("poisson_tol", ctypes.c_double), ("poisson_max_iter", ctypes.c_int32),
        ("poisson_min_iter", ctypes.c_int32), ("poisson_fixed_iter", ctypes.c_int32),
        ("poisson_loop", ctypes.c_int32), ("start_step", ctypes.c_int64),
        ("tile_rows", ctypes.c_int32), ("potential_scheme", ctypes.c_int32),
        ("chi", ctypes.c_double), ("field_mode", ctypes.c_int32),
        ("lagged_field", ctypes.c_int32),
    ]

    @classmethod
    def from_dict(cls, d):
        p = cls()
        for name, _ in cls._fields_:
            if name in d:
                setattr(p, name, d[name])
        return p


class Stats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("steps", ctypes.c_int32),
        ("poisson_iters_total", ctypes.c_int32), ("poisson_iters_min", ctypes.c_int32),
        ("poisson_iters_max", ctypes.c_int32), ("not_converged_steps", ctypes.c_int32),
        ("nonfinite", ctypes.c_int32), ("last_rel_change", ctypes.c_double),
        ("sum_phi", ctypes.c_double), ("sum_q", ctypes.c_double),
        ("kernel_launches", ctypes.c_int64),
    ]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class KernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_int64 * 4)]

    KINDS = ("moments", "potential", "potential_idle", "coupled")

    def as_dict(self):
        return {k: {"ms": self.ms[j], "launches": self.launches[j]}
                for j, k in enumerate(self.KINDS)}


class SlotStatus(ctypes.Structure):
    _fields_ = [
        ("slot", ctypes.c_int32), ("live", ctypes.c_int32), ("request_id", ctypes.c_int64),
        ("steps", ctypes.c_int64), ("poisson_iters", ctypes.c_int64),
        ("steady", ctypes.c_int32), ("capped", ctypes.c_int32), ("status", ctypes.c_int32),
        ("pad", ctypes.c_int32), ("rel_change_phi", ctypes.c_double),
        ("rel_change_u", ctypes.c_double),
    ]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "pad"}


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("live_slots", ctypes.c_int32), ("max_slots", ctypes.c_int32),
        ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
        ("tiles_used", ctypes.c_int32), ("tile_capacity", ctypes.c_int32),
        ("steps_run", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("tile_rows", ctypes.c_int32), ("steps_per_graph", ctypes.c_int32),
    ]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None

# name -> (restype, argtypes); every function declared in include/ehd.h
SIGNATURES = {
    "ehd_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]),
    "ehd_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "ehd_set_fields": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5 + [ctypes.c_int]),
    "ehd_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Stats)]),
    "ehd_read_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "ehd_loop_kind": (ctypes.c_int, [ctypes.c_void_p]),
    "ehd_solve_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]),
    "ehd_read_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "ehd_contact_line": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double,
                                        ctypes.POINTER(ctypes.c_double)]),
    "ehd_diag_index_errors": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]),
    "ehd_state_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "ehd_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "ehd_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "ehd_diag_expire_barrier": (ctypes.c_int, [ctypes.c_void_p]),
    "ehd_destroy": (None, [ctypes.c_void_p]),
    "ehd_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ehd_version": (ctypes.c_char_p, []),
    "ehd_abi_sizes": (ctypes.c_int, [ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "ehd_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ehd_batch_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "ehd_batch_admit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Params)]
                        + [ctypes.c_void_p] * 4 + [ctypes.c_int64, ctypes.POINTER(ctypes.c_int)]),
    "ehd_batch_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "ehd_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ehd_batch_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(SlotStatus), ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "ehd_batch_read_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint,
                                             ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "ehd_batch_retire": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ehd_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchInfo)]),
    "ehd_batch_destroy": (None, [ctypes.c_void_p]),
    "ehd_potential_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.POINTER(ctypes.c_int),
                                                   ctypes.POINTER(ctypes.c_double)]),
    "ehd_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KernelTimes)]),
    "ehd_diag_smem_bandwidth": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "ehd_diag_grid_exchange": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double)]),
    "ehd_use_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "ehd_slabs_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "ehd_slabs_set_fields": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 5),
    "ehd_slabs_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Stats)]),
    "ehd_slabs_read_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint,
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "ehd_slabs_exchange_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "ehd_slabs_destroy": (None, [ctypes.c_void_p]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2407_01654_gb300.build`"
                " (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, what):
    if code != EHD_OK:
        raise EhdError(code, what)


def _host(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def smem_bandwidth(stream=None):
    """Shared-memory bandwidth of the current device in bytes per second (loads plus
    stores, measured by ehd_diag_smem_bandwidth)."""
    v = ctypes.c_double()
    _check(lib().ehd_diag_smem_bandwidth(stream, ctypes.byref(v)), "ehd_diag_smem_bandwidth")
    return v.value


def grid_exchange_floor(nx, ny, stream=None):
    """Seconds per cycle of the two-step on-chip loop's exchange alone (band export, grid
    barrier, ring import; no arithmetic) on an nx x ny lattice of 64 x 56 tiles, measured by
    ehd_diag_grid_exchange."""
    v = ctypes.c_double()
    _check(lib().ehd_diag_grid_exchange(stream, int(nx), int(ny), ctypes.byref(v)),
           "ehd_diag_grid_exchange")
    return v.value


def output_pointers(outs, shape, device):
    """Addresses of caller-owned output buffers for ehd_read_fields, after checking that
    each has the shape and type the call writes: C-contiguous numpy float64 on the host,
    contiguous float32 CUDA tensors for device reads.  Raises ValueError otherwise."""
    ptrs = []
    for o in outs:
        if device:
            if not (_is_torch_cuda(o) and str(o.dtype) == "torch.float32"
                    and tuple(o.shape) == tuple(shape) and o.is_contiguous()):
                raise ValueError("device outputs must be contiguous float32 CUDA tensors "
                                 f"of shape {tuple(shape)}")
            ptrs.append(o.data_ptr())
        else:
            if not (isinstance(o, np.ndarray) and o.dtype == np.float64
                    and o.shape == tuple(shape) and o.flags.c_contiguous and o.flags.writeable):
                raise ValueError("host outputs must be writeable C-contiguous float64 arrays "
                                 f"of shape {tuple(shape)}")
            ptrs.append(o.ctypes.data)
    return ptrs


class Sim:
    """One simulation on the GPU.

    params: dict of ehd_params fields (see paper_2407_01654_gb300.workloads).
    workspace: "torch" (a torch uint8 tensor owned by this object), "library" (the
    library allocates), or a torch tensor / (pointer, bytes) pair supplied by the caller.
    stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (torch's current
    stream when torch is used, else the default stream).
    """

    def __init__(self, params, workspace="torch", stream=None):
        L = lib()
        self.params = dict(params)
        self._p = Params.from_dict(self.params)
        nb = ctypes.c_size_t()
        _check(L.ehd_workspace_bytes(ctypes.byref(self._p), ctypes.byref(nb)), "ehd_workspace_bytes")
        self.workspace_bytes = nb.value
        self._ws_keep = None
        ptr = None
        if isinstance(workspace, str) and workspace == "torch":
            import torch
            self._ws_keep = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._ws_keep.data_ptr() + 255) // 256 * 256
        elif isinstance(workspace, str) and workspace == "library":
            ptr = None
        elif isinstance(workspace, tuple):
            ptr = workspace[0]
        elif workspace is not None:
            self._ws_keep = workspace
            ptr = workspace.data_ptr()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        h = ctypes.c_void_p()
        _check(L.ehd_create(ctypes.byref(self._p), ptr, nb.value, self.stream, ctypes.byref(h)),
               "ehd_create")
        self._h = h
        self.nx, self.ny = self.params["nx"], self.params["ny"]

    # -- life cycle ----------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().ehd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -----------------------------------------------------------------------
    def set_fields(self, phi, q, ux, uy, p=None):
        """Host numpy arrays (converted to double) or CUDA float32 torch tensors."""
        arrs = [phi, q, ux, uy] + ([p] if p is not None else [])
        if _is_torch_cuda(phi):
            keep = [a.contiguous() for a in arrs]
            ptrs = [a.data_ptr() for a in keep]
            mem = EHD_DEVICE
        else:
            keep = [_host(a) for a in arrs]
            ptrs = [a.ctypes.data for a in keep]
            mem = EHD_HOST
        if p is None:
            ptrs.append(None)
        code = lib().ehd_set_fields(self._h, *ptrs, mem)
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_set_fields")
        return code

    def step(self, nsteps=1, stats=True):
        st = Stats()
        code = lib().ehd_step(self._h, int(nsteps), ctypes.byref(st) if stats else None)
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_step")
        out = st.as_dict() if stats else {}
        out["status"] = code
        return out

    def use_graphs(self, enable=True):
        """enable=False: later steps queue their kernels one by one from the host instead of
        launching captured graphs (same states, bit for bit)."""
        _check(lib().ehd_use_graphs(self._h, 1 if enable else 0), "ehd_use_graphs")

    def diag_expire_barrier(self):
        """Diagnostics: the next on-chip potential solve's grid barrier never completes, so
        its bounded waits run out and the call reports EHD_ERR_TIMEOUT (9)."""
        _check(lib().ehd_diag_expire_barrier(self._h), "ehd_diag_expire_barrier")

    def loop_kind(self):
        """1 streaming loop, 2 on-chip loop, 3 / 4 on-chip loop with two / three
        sub-iterations per exchange."""
        return int(lib().ehd_loop_kind(self._h))

    def uses_resident_loop(self):
        """True when the potential loop runs on chip (one cooperative launch per solve)."""
        return self.loop_kind() in (2, 3, 4)

    def read_stats(self):
        st = Stats()
        code = lib().ehd_read_stats(self._h, ctypes.byref(st))
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_read_stats")
        out = st.as_dict()
        out["status"] = code
        return out

    def solve_potential(self, tol=0.0, max_iter=0):
        it = ctypes.c_int()
        rel = ctypes.c_double()
        code = lib().ehd_solve_potential(self._h, float(tol), int(max_iter), ctypes.byref(it),
                                         ctypes.byref(rel))
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_solve_potential")
        return it.value, rel.value, code

    def read_fields(self, names=FIELDS, device=False, out=None):
        """dict name -> numpy float64 array [ny, nx] (or torch float32 CUDA tensors).
        out: optional dict name -> caller-owned array of that shape and type (C-contiguous
        numpy float64 on the host, contiguous float32 CUDA tensors with device=True) that
        the library writes into, so that repeated reads reuse their buffers; it must hold
        every requested field."""
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        if out is not None:
            outs = [out[n] for n in order]
            ptrs = output_pointers(outs, (self.ny, self.nx), device)
        elif device:
            import torch
            outs = [torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda")
                    for _ in order]
            ptrs = [o.data_ptr() for o in outs]
        else:
            outs = [np.empty((self.ny, self.nx), dtype=np.float64) for _ in order]
            ptrs = [o.ctypes.data for o in outs]
        mem = EHD_DEVICE if device else EHD_HOST
        arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
        _check(lib().ehd_read_fields(self._h, mask, arr, mem), "ehd_read_fields")
        return dict(zip(order, outs))

    def contact_line(self, level=0.5):
        """Contact line of a drop on the bottom wall: dict left, right, radius (lattice
        units; NaN when there is none or it crosses the periodic seam)."""
        out = (ctypes.c_double * 3)()
        _check(lib().ehd_contact_line(self._h, float(level), out), "ehd_contact_line")
        return {"left": out[0], "right": out[1], "radius": out[2]}

    def index_errors(self):
        """Out-of-range indices the index-checking build met (always 0 otherwise)."""
        n = ctypes.c_uint()
        _check(lib().ehd_diag_index_errors(self._h, ctypes.byref(n)), "ehd_diag_index_errors")
        return n.value

    def contact_radius_history(self, total_steps, every, level=0.5):
        """Runs total_steps steps and returns [(steps run, radius)] of the contact line on
        the bottom wall, at the start and after every `every` steps (the histories of Sec.
        7.2, Fig. 11, normalise radius by its first value)."""
        out = [(0, self.contact_line(level)["radius"])]
        done = 0
        while done < total_steps:
            n = min(every, total_steps - done)
            self.step(n, stats=False)
            done += n
            out.append((done, self.contact_line(level)["radius"]))
        return out

    def profile(self, enable=True):
        _check(lib().ehd_profile(self._h, 1 if enable else 0), "ehd_profile")

    def profile_read(self):
        kt = KernelTimes()
        _check(lib().ehd_profile_read(self._h, ctypes.byref(kt)), "ehd_profile_read")
        return kt.as_dict()

    def save_state(self):
        nb = ctypes.c_size_t()
        _check(lib().ehd_state_bytes(self._h, ctypes.byref(nb)), "ehd_state_bytes")
        buf = ctypes.create_string_buffer(nb.value)
        _check(lib().ehd_save_state(self._h, buf, nb.value), "ehd_save_state")
        return buf.raw

    def load_state(self, blob):
        """blob: bytes from save_state, or a host uint8 torch tensor holding them (e.g. in
        pinned memory, passed to the library without a copy)."""
        if hasattr(blob, "data_ptr"):
            _check(lib().ehd_load_state(self._h, ctypes.c_void_p(blob.data_ptr()), blob.numel()),
                   "ehd_load_state")
            return
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().ehd_load_state(self._h, buf, len(blob)), "ehd_load_state")


class Slabs:
    """One lattice computed by `nslabs` slabs of rows with their own buffers, exchanging
    the rows that cross each cut (the ehd_slabs_* calls).  Host numpy I/O only."""

    def __init__(self, params, nslabs, stream=None):
        self.ny, self.nx = int(params["ny"]), int(params["nx"])
        self._p = Params.from_dict(params)
        h = ctypes.c_void_p()
        _check(lib().ehd_slabs_create(ctypes.byref(self._p), int(nslabs), stream, ctypes.byref(h)),
               "ehd_slabs_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().ehd_slabs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, phi, q, ux, uy, p=None):
        arrs = [_host(a) for a in (phi, q, ux, uy)] + ([_host(p)] if p is not None else [])
        ptrs = [a.ctypes.data for a in arrs] + ([None] if p is None else [])
        code = lib().ehd_slabs_set_fields(self._h, *ptrs)
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_slabs_set_fields")
        return code

    def step(self, nsteps=1):
        st = Stats()
        code = lib().ehd_slabs_step(self._h, int(nsteps), ctypes.byref(st))
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_slabs_step")
        out = st.as_dict()
        out["status"] = code
        return out

    def read_fields(self, names=FIELDS):
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        outs = [np.empty((self.ny, self.nx), dtype=np.float64) for _ in order]
        arr = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
        _check(lib().ehd_slabs_read_fields(self._h, mask, arr), "ehd_slabs_read_fields")
        return dict(zip(order, outs))

    def exchange_bytes(self):
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().ehd_slabs_exchange_bytes(self._h, ctypes.byref(a), ctypes.byref(b)),
               "ehd_slabs_exchange_bytes")
        return a.value, b.value


class Batch:
    """Many simulations resident in one device-memory arena (the ehd_batch_* calls).

    hbm_budget: bytes of the arena; max_slots: concurrent requests; steady_tol: relative L2
    change of phi and u over one run call below which a slot is steady; step_cap: steps
    after which a slot is reported capped.  arena: "torch" (a torch uint8 tensor owned by
    this object) or "library"."""

    def __init__(self, hbm_budget, max_slots=64, steady_tol=1e-6, step_cap=300000,
                 arena="torch", stream=None):
        L = lib()
        self._keep = None
        ptr = None
        if arena == "torch":
            import torch
            self._keep = torch.empty(int(hbm_budget) + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._keep.data_ptr() + 255) // 256 * 256
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = ctypes.c_void_p()
        _check(L.ehd_batch_create(int(hbm_budget), int(max_slots), float(steady_tol),
                                  int(step_cap), ptr, int(stream), ctypes.byref(h)),
               "ehd_batch_create")
        self._h = h
        self.max_slots = max_slots
        self.shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().ehd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, params, fields, request_id=0):
        """Returns the slot index, or None when the batch is full (EHD_ERR_BUSY)."""
        p = Params.from_dict(params)
        arrs = [_host(fields[k]) for k in ("phi", "q", "ux", "uy")]
        slot = ctypes.c_int(-1)
        code = lib().ehd_batch_admit(self._h, ctypes.byref(p), *[a.ctypes.data for a in arrs],
                                     int(request_id), ctypes.byref(slot))
        if code == 6:
            return None
        if code not in (EHD_OK, 4):
            _check(code, "ehd_batch_admit")
        self.shapes[slot.value] = (params["ny"], params["nx"])
        return slot.value

    def set_schedule(self, tile_rows=32, steps_per_graph=16):
        """Tile height of every slot's potential loop and steps per captured graph; only
        while no slot is live.  Returns False when slots are live (EHD_ERR_BUSY)."""
        code = lib().ehd_batch_set_schedule(self._h, int(tile_rows), int(steps_per_graph))
        if code == 6:
            return False
        _check(code, "ehd_batch_set_schedule")
        return True

    def run(self, nsteps):
        code = lib().ehd_batch_run(self._h, int(nsteps))
        if code not in (EHD_OK, 4, 5):
            _check(code, "ehd_batch_run")
        return code

    def poll(self):
        arr = (SlotStatus * self.max_slots)()
        n = ctypes.c_int()
        _check(lib().ehd_batch_poll(self._h, arr, self.max_slots, ctypes.byref(n)), "ehd_batch_poll")
        return [arr[i].as_dict() for i in range(n.value)]

    def read_fields(self, slot, names=FIELDS):
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        shape = self.shapes[slot]
        outs = [np.empty(shape, dtype=np.float64) for _ in order]
        ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
        _check(lib().ehd_batch_read_fields(self._h, int(slot), mask, ptrs, EHD_HOST),
               "ehd_batch_read_fields")
        return dict(zip(order, outs))

    def retire(self, slot):
        _check(lib().ehd_batch_retire(self._h, int(slot)), "ehd_batch_retire")
        self.shapes.pop(slot, None)

    def info(self):
        bi = BatchInfo()
        _check(lib().ehd_batch_info(self._h, ctypes.byref(bi)), "ehd_batch_info")
        return bi.as_dict()
