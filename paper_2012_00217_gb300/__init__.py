"""GB300 (sm_103a) library for the matrix-free MBL eigensolver hot path.

The compute runs in the CUDA library built from ``csrc/`` (see ``build.py``) and
exposed through the C ABI in ``include/mbl.h``; ``binding`` is its ctypes
marshalling layer.  PyTorch supplies device memory and streams only.
"""
from . import binding  # noqa: F401
from .binding import (MODE_FP64, MODE_MIXED, MBLError, basis_build, basis_rank,  # noqa: F401
                      basis_size, bounds_workspace_size, entanglement_entropy, gap_ratio,
                      hamiltonian_apply, lobpcg_solve,
                      lobpcg_workspace_size, make_chain, make_opts, spectrum_bounds)
