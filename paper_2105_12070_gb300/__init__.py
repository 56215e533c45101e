"""GB300-native batched finite-rate chemistry solve (Morev et al., arXiv 2105.12070, Sec. 2.1-2.3).

The compute path is the CUDA library libchemgpu.so (C ABI in include/chemgpu.h); `chem` is its
thin Python binding, `autograd` wraps the discrete adjoint in a torch.autograd.Function, `ranks`
holds the multi-process helpers, `autotune` picks launch shapes, `phases` prints the kernel's
per-phase cycle counters, and `synth` draws the seeded synthetic inputs.
"""
from .chem import (ChemError, ChemOpts, ChemStats, Mechanism, chem_adjoint, chem_describe_mechanism,  # noqa: F401
                   chem_get_lnA,
                   chem_integrate, chem_integrate_mapped, chem_integrate_noalloc, chem_integrate_record,
                   chem_integrate_varp, chem_jacobian, chem_last_cell_counters, chem_load_mechanism, chem_rates,
                   chem_set_lnA, default_opts, load_library)
