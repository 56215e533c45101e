// Internal interface of the discrete-adjoint kernels (adjoint.cu) for the C ABI in
// chem_kernels.cu.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "chem_internal.h"

namespace chemgpu {

// Device workspace (doubles) the reverse sweep needs for ncells cells besides the caller's
// arrays: the per-cell ln A gradients when the caller keeps none, and the partial sums of the
// fixed-order reduction over cells.
size_t adjoint_workspace_doubles(int R, int64_t ncells, bool have_cell_grads);

// Enqueue the reverse sweep on `st` (see chem_adjoint in chemgpu.h for the arrays).  p_cgs in
// dyn/cm^2.  ws: adjoint_workspace_doubles(..) doubles; counters: 2 ints of device memory.
// Returns a CHEM_* code, with a message in err on failure.
int adjoint_enqueue(const DevMech& d, int num_sms, size_t max_smem, double p_cgs, int64_t ncells, const double* rec,
                    int rec_cap, const int32_t* nsteps, const int32_t* status, const double* gT, const double* gY,
                    double* gT0, double* gY0, double* g_lnA, double* g_lnA_cells, double* ws, int* counters,
                    cudaStream_t st, std::string& err);

}  // namespace chemgpu
