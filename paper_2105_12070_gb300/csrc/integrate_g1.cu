// The integrate kernels (Rosenbrock and Seulex) for cell groups of 1 warp, and their launchers.
#include "integrate_device.cuh"

CHEM_DEFINE_INTEGRATE_LAUNCHERS(1)
