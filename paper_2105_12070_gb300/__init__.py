"""GB300-native batched finite-rate chemistry solve (Morev et al., arXiv 2105.12070, Sec. 2.1-2.3).

The compute path is the CUDA library libchemgpu.so (C ABI in include/chemgpu.h); `chem` is its
thin Python binding and `synth` draws the seeded synthetic inputs.
"""
from .chem import (ChemError, ChemOpts, ChemStats, Mechanism, chem_integrate, chem_jacobian,  # noqa: F401
                   chem_last_cell_counters, chem_load_mechanism, chem_rates, default_opts, load_library)
