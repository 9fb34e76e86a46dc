"""GB300-native coupled phase-field lattice Boltzmann step for two-phase EHD
(arXiv 2407.01654).  The compute path is the CUDA library behind the C ABI in
include/ehd.h; `paper_2407_01654_gb300.ehd` is its thin ctypes binding."""
