"""GB300 (sm_103a) coupled flow + substrate-transport lattice Boltzmann solvers of the microbial
fuel cell model of Tsompanas et al. (arXiv 1802.07525).

The compute path is the CUDA library ``_lib/libmfc.so`` behind the C ABI of ``include/mfc.h``;
:mod:`paper_1802_07525_gb300.mfc` is its thin ctypes binding.
"""
from .mfc import (EXPORTED, Lattice, MfcError, SolveResult, lattice_bytes, lib, make_desc,  # noqa: F401
                  make_params, status_string)
from .mfc import *  # noqa: F401,F403
