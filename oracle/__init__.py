"""CPU oracle (FP64, numpy) of the coupled phase-field LB step for two-phase EHD.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg.  The library never imports it and shares no code with it.
"""
from .ehd import Params, Sim, StepStats  # noqa: F401
