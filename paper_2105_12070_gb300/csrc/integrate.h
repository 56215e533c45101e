// Internal interface between the host side of the library (chem_kernels.cu) and the integrate
// kernels, which are compiled in one translation unit per cell-group width G (integrate_g*.cu)
// so that the build runs in parallel.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "chem_internal.h"

// Threads per CTA of the integrate kernels (8 warps: with ~230 registers per thread that is the
// register file, and shared memory holds 4 cells of 53 species)
#ifndef CHEM_MAX_THREADS_PER_CTA
#define CHEM_MAX_THREADS_PER_CTA 256
#endif

namespace chemgpu {

// Arguments of one integrate launch (all pointers device memory).
struct IntegrateArgs {
  double p, dt, rtol, atol;
  double *T, *Y;
  double* h_inout;
  int32_t* status;
  int32_t* steps_out;
  int32_t* rej_out;
  unsigned long long* totals;  // steps, rejects, failed cells, refine fallbacks
  int* queue;
  int64_t ncells;     // number of cells in the arrays (the stride of Y)
  int64_t first;      // this launch integrates cells first .. first + count - 1
  int64_t count;
  int max_steps;
  int use_queue;
  int mixed;          // 0: FP64 factors; 1: FP32 factors, 2: FP32 pairs (+ FP64-residual refinement)
  int refine_sweeps;  // refinement sweeps per stage solve (mixed)
  double* rec;        // record mode: checkpoint of every accepted step (NULL: off)
  int rec_cap;        // checkpoints per cell
  int solver;         // CHEM_SOLVER_*
  int fdjac;          // forward-difference Jacobian instead of the analytical one
  const double* p_cells;  // per-cell pressure in Pa (NULL: p for every cell)
  unsigned long long* phase;  // per-phase cycle counters (builds with CHEM_PHASE_TIMERS; else NULL)
};
// The integrate kernel of one group width (G = 1, 2, 4 or 8 warps per cell) and solver
// (CHEM_SOLVER_*), for occupancy queries and attributes; NULL for another G.
const void* integrate_kernel_fn(int G, int solver);

// Launches it: grid CTAs of `threads` threads with `smem` bytes of dynamic shared memory each,
// the per-cell plan of make_plan(K, R, n_pd, G).
void integrate_launch(int G, int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                      const IntegrateArgs& a);

// One translation unit per G defines these.
const void* integrate_kernel_fn_g1(int solver);
const void* integrate_kernel_fn_g2(int solver);
const void* integrate_kernel_fn_g4(int solver);
const void* integrate_kernel_fn_g8(int solver);
void integrate_launch_g1(int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                         const IntegrateArgs& a);
void integrate_launch_g2(int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                         const IntegrateArgs& a);
void integrate_launch_g4(int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                         const IntegrateArgs& a);
void integrate_launch_g8(int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                         const IntegrateArgs& a);

}  // namespace chemgpu
