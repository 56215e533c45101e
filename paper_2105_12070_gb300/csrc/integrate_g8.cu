// The integrate kernels (Rosenbrock and Seulex) for cell groups of 8 warps, and their launchers.
#include "integrate_device.cuh"

CHEM_DEFINE_INTEGRATE_LAUNCHERS(8)
