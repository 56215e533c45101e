/*
 * chemgpu: GB300 (sm_103a) batched finite-rate chemistry solve -- C ABI.
 *
 * The operation (Morev et al., "Fast reactive flow simulations using analytical Jacobian and
 * dynamic load balancing in OpenFOAM"): for every CFD cell, integrate the stiff
 * constant-pressure ideal-gas system d(phi)/dt = f(phi), phi = [T, Y_1 .. Y_{K-1}]
 * (Sec. 2.1, Eq. 1), over one flow time step dt, with a linearly implicit method (Sec. 2.3,
 * Eq. 2) in adaptive Rosenbrock form, using the analytical Jacobian of f and a dense LU of the
 * iteration matrix (Sec. 2.3).  Y_K = 1 - sum of the others (Eq. 1).
 *
 * Conventions shared by all entry points
 *   - Units at the boundary: T in K, p in Pa, dt in s, mass fractions dimensionless; internal
 *     arithmetic is cgs.  The rate outputs are in K/s and 1/s.
 *   - Cell arrays are species-major: Y[k * ncells + c] for species k of cell c, all K species.
 *   - Array pointers may be device pointers (the call is asynchronous on `stream`, results valid
 *     after the stream is synchronised) or host pointers, pageable or pinned (the library copies
 *     through its own device workspace with cudaMemcpyAsync on `stream`, then synchronises the
 *     stream before returning).  All arrays of one call must be of the same kind.  The caller
 *     owns every array; the library owns the mechanism handle and its workspaces.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - Return value: 0 on success; a negative CHEM_E* code on invalid arguments or a CUDA error,
 *     with a message in chem_last_error() (thread-local).  No exception crosses the ABI and no
 *     kernel traps: per-cell numerical failure is reported in status[], not as a call failure.
 *   - A mechanism handle may be used from one host thread at a time.
 */
#ifndef CHEMGPU_H
#define CHEMGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define CHEM_OK 0
#define CHEM_EINVAL (-1)   /* bad argument (NULL, ncells < 0, dt <= 0, rtol <= 0, ...) */
#define CHEM_EFILE (-2)    /* mechanism file unreadable or malformed */
#define CHEM_ECUDA (-3)    /* a CUDA runtime call failed */
#define CHEM_ESIZE (-4)    /* mechanism too large for the kernels' shared-memory plan */

/* per-cell status written by chem_integrate (the cell keeps its last accepted state) */
#define CHEM_CELL_OK 0
#define CHEM_CELL_MAX_STEPS 1    /* step-attempt limit reached before t = dt */
#define CHEM_CELL_H_UNDERFLOW 2  /* proposed step fell below 1e-14 dt */
#define CHEM_CELL_BAD_INPUT 3    /* non-finite input or T <= 0; state left unchanged */
#define CHEM_CELL_RECORD_FULL 4  /* chem_integrate_record: more accepted steps than max_steps_rec;
                                    the cell stops at its last recorded step */

/* integrators (chem_opts.solver) */
#define CHEM_SOLVER_ROSENBROCK 0 /* 4-stage L-stable Rosenbrock method, order 4(3) (default) */
#define CHEM_SOLVER_SEULEX 1     /* the paper's Seulex (Sec. 2.3): linearly implicit Euler with
                                    extrapolation, harmonic step-number sequence, up to 8 columns,
                                    order and step chosen by work per unit step; FP64 only */

/* Jacobian of the Rosenbrock solve (chem_opts.jacobian) */
#define CHEM_JAC_ANALYTIC 0 /* the analytical Jacobian (Sec. 2.3; default) */
#define CHEM_JAC_FD 1       /* first-order forward differences, N + 1 rate evaluations: the
                               alternative the paper measures the analytical Jacobian against */

/* precision of the linear solves inside the Rosenbrock stages (chem_opts.precision) */
#define CHEM_PREC_FP64 0     /* FP64 LU and substitutions */
#define CHEM_PREC_MIXED 1    /* FP32 LU + FP64-residual iterative refinement; rates, Kc, error
                                norm, step control and state update stay FP64 */
#define CHEM_PREC_MIXED_FF 2 /* LU and substitutions in FP32 pairs (hi + lo, ~48 significand
                                bits in FP32 arithmetic) + FP64-residual iterative refinement
                                (refine_sweeps 0 takes the pair solve without refinement);
                                the rest FP64 as for CHEM_PREC_MIXED */

typedef struct chem_mech chem_mech; /* opaque */

typedef struct {
  int precision;     /* CHEM_PREC_FP64 (default), CHEM_PREC_MIXED or CHEM_PREC_MIXED_FF */
  int refine_sweeps; /* mixed: FP64-residual refinement sweeps per stage solve (default 2;
                        1..4 for CHEM_PREC_MIXED, 0..4 for CHEM_PREC_MIXED_FF) */
  int max_steps;     /* step attempts per cell per call (default 100000) */
  int use_queue;     /* 1 (default): persistent kernel pulling cells from a device work queue;
                        0: static round-robin assignment of cells to warps */
  int cells_per_cta; /* cells in flight per CTA; 0 = automatic */
  int ctas_per_sm;   /* resident CTAs per SM for the persistent grid; 0 = automatic */
  int warps_per_cell; /* 1, 2, 4 or 8 warps cooperate on one cell; 0 = automatic */
  int use_graph;      /* 1: launch through a CUDA graph that the library captures once for this
                         exact argument set and replays on identical calls (host arrays: the
                         graph holds the launches on the library's staging buffers, the copies
                         stay outside it); 0 (default): direct launches */
  int batch_cells;    /* > 0: split the cells into consecutive batches of this many cells, one
                         kernel launch per batch (the one-launch-per-batch comparison of the
                         persistent queue); 0 (default): one launch for all cells */
  int solver;         /* CHEM_SOLVER_ROSENBROCK (default) or CHEM_SOLVER_SEULEX */
  int jacobian;       /* CHEM_JAC_ANALYTIC (default) or CHEM_JAC_FD (Rosenbrock only) */
} chem_opts;

typedef struct {
  int64_t steps;        /* accepted steps, summed over cells */
  int64_t rejects;      /* rejected step attempts */
  int64_t failed_cells; /* cells whose status is not CHEM_CELL_OK */
  int64_t refine_fallbacks; /* mixed precision: stage solves that fell back to an FP64 factor */
  double kernel_ms;     /* device time of the call's integrate launches in milliseconds: CUDA events
                           on `stream` around them, after any host-to-device staging and before the
                           copy back (chem_integrate and the entry points built on it; 0 from
                           chem_integrate_noalloc, which records no events) */
} chem_stats;

/* Fill `opts` with the defaults. */
void chem_default_opts(chem_opts* opts);

/* Load a mechanism file and upload its tables to the current CUDA device.  Two formats:
 *   - CHEMMECH (the first non-comment line starts with that word): the text format of the
 *     synthetic generator -- elements, species with molar mass and NASA 7-coefficient
 *     polynomials, reversible reactions of type elementary, third-body, Lindemann or Troe
 *     fall-off;
 *   - anything else is read as CHEMKIN-II (ELEMENTS, SPECIES, THERMO with NASA-7 cards,
 *     REACTIONS with unit keywords, reversible '=' / '<=>', integer coefficients, '+M' with
 *     efficiencies, '(+M)' with LOW and TROE, a named third body '(+AR)' (efficiency 1 for it,
 *     0 for the others), DUPLICATE).  Forms the kernels do not hold are refused with
 *     CHEM_EFILE and a message: irreversible '=>', REV, PLOG, SRI, HIGH, FORD/RORD, more than
 *     two molecules on a side.
 * The file is parsed before the GPU is touched (a malformed file gives CHEM_EFILE on any
 * machine).  On success *out owns the tables until chem_free_mechanism. */
int chem_load_mechanism(const char* path, chem_mech** out);
void chem_free_mechanism(chem_mech* mech);

/* Parse a mechanism file on the host (no GPU needed) and write the tables the kernels would use,
 * in file order, as text: "species K", one line per species "sp W Tmid a_low[7] a_high[7]",
 * "reactions R", one line per reaction "rx type n_reac reac.. n_prod prod.. A b Ea/R [eff K
 * values] [low A0 b0 Ea0/R] [troe alpha T3 T1 T2]" (species indices ascending within a side;
 * type 0 elementary, 1 third-body, 2 Lindemann, 3 Troe; Ea/R in K; a missing Troe T2 is 1e30).
 * *need receives the size including the terminating NUL; cap <= 0 only queries it, a smaller
 * positive cap gives CHEM_ESIZE.  For checking the reader against an independent one. */
int chem_describe_mechanism(const char* path, char* buf, int64_t cap, int64_t* need);

/* Number of species K (= state length N) and reactions R. */
int chem_mech_dims(const chem_mech* mech, int* K, int* R);

/* Reaction-type counts of a loaded mechanism: plain third-body reactions and fall-off
 * (Lindemann or Troe) reactions; their sum is the number of pressure-dependent reactions, which
 * sets the size of the per-cell working set with K and R.  Either pointer may be NULL. */
int chem_mech_counts(const chem_mech* mech, int* n_third_body, int* n_falloff);

/* Source term f of Eq. 1 for ncells cells at pressure p_Pa:
 *   dPhidt[0 * ncells + c] = dT/dt, dPhidt[(1 + k) * ncells + c] = dY_k/dt for k < K-1.
 * T[ncells], Y[K * ncells] as above (Y_K is recomputed as 1 - sum of the others). */
int chem_rates(const chem_mech* mech, double p_Pa, const double* T, const double* Y, int64_t ncells,
               double* dPhidt, void* stream);

/* Analytical Jacobian J = df/dphi (Sec. 2.3) for ncells cells:
 *   J[c * N * N + i * N + j] = d f_i / d phi_j, phi = [T, Y_1 .. Y_{K-1}], N = K. */
int chem_jacobian(const chem_mech* mech, double p_Pa, const double* T, const double* Y, int64_t ncells,
                  double* J, void* stream);

/* Integrate every cell over [0, dt] (Sec. 2.1 Eq. 1; Sec. 2.3 Eq. 2 and the adaptive sub-steps
 * with carry-over).  T[ncells] and Y[K * ncells] are read and overwritten with the state at dt.
 * h_inout[ncells] (may be NULL): on entry a positive value is the first sub-step to try
 * (else 0.01 dt); on exit the controller's next proposed sub-step, for the next call.
 * status[ncells] (may be NULL): CHEM_CELL_* per cell.
 * opts may be NULL (defaults); stats may be NULL; when given, the call synchronises `stream`
 * to read the totals back. */
int chem_integrate(const chem_mech* mech, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                   double rtol, double atol, double* h_inout, int32_t* status, const chem_opts* opts,
                   chem_stats* stats, void* stream);

/* chem_integrate without any device-memory allocation.  The paper has no counterpart: this
 * entry point serves callers that cannot call cudaMalloc while they run, for instance a flow
 * solver that reserves all device memory for its own pool at start-up, or a time loop that must
 * not pay the device-wide synchronisation cudaMalloc / cudaFree can cause.
 *
 * Same arguments and results as chem_integrate, plus optional device arrays steps[ncells] and
 * rejects[ncells] for the per-cell counters.  Differences:
 *   - every array must be device memory (host arrays would need a staging buffer):
 *     CHEM_EINVAL otherwise;
 *   - the work-queue counter, the call totals and the per-cell counters live in one fixed
 *     2 MiB array inside the library (static device memory, loaded with the library on every
 *     GPU that uses it and held until the process exits), so at most 262144 cells per call:
 *     larger calls return CHEM_ESIZE without launching anything;
 *   - the library looks the array's device address up the first time the entry point runs on a
 *     device (cudaGetSymbolAddress), so make that first call before any stream capture;
 *   - all calls share that array: it is reset at the start of each call, and two calls whose
 *     work overlaps on the GPU (different streams, no ordering between them) race on it;
 *   - opts->batch_cells and opts->use_graph are ignored: the call is always one launch over all
 *     cells, enqueued directly on `stream` (no library-owned CUDA graph, which would allocate);
 *   - the per-cell counters go to steps / rejects only: chem_last_cell_counters keeps reporting
 *     the last chem_integrate on the handle.
 * It allocates nothing itself; the mechanism handle, loaded beforehand, owns its tables. */
int chem_integrate_noalloc(const chem_mech* mech, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                           double rtol, double atol, double* h_inout, int32_t* status, int32_t* steps,
                           int32_t* rejects, const chem_opts* opts, chem_stats* stats, void* stream);

/* chem_integrate with a pressure per cell: p_Pa[ncells] (Pa) instead of one value, for flow
 * solvers whose cells sit at different pressures (the constant-pressure system of Eq. 1 holds
 * within each cell over dt).  Device arrays only.  A cell whose pressure is not positive and
 * finite reports CHEM_CELL_BAD_INPUT. */
int chem_integrate_varp(const chem_mech* mech, const double* p_Pa, double* T, double* Y, int64_t ncells, double dt,
                        double rtol, double atol, double* h_inout, int32_t* status, const chem_opts* opts,
                        chem_stats* stats, void* stream);

/* chem_integrate with zonal reference-cell mapping (DLBFoam's, Sec. 2.2): a cell whose state
 * lies within |T - T_r| <= tol_T and max_k |Y_k - Y_r,k| <= tol_Y of reference state r (an ambient
 * zone of low reactivity; the first such r) is not solved: it receives that reference's change
 * over dt, T += T_r(dt) - T_r, Y_k += Y_r,k(dt) - Y_r,k (k < K-1), Y_K = 1 - sum, and the
 * reference's status.  The other cells and the references are solved together by chem_integrate
 * (references from a cold start; a solved cell keeps its h_inout carry-over, a mapped cell's is
 * left unchanged).
 *   refs[n_ref][1 + K] (HOST array, n_ref <= 64): T_r, Y_r,0 .. Y_r,K-1;
 *   zone[ncells] (device, may be NULL): the reference a cell was mapped to, or -1 if solved;
 *   *n_mapped (host, may be NULL): the number of mapped cells.
 * The other arrays are device arrays as for chem_integrate.  The call synchronises `stream` once
 * (after classifying, to size the solve); opts->use_graph is ignored.  The paper has no
 * formulas for the mapping; the zone test is this library's reading of it. */
int chem_integrate_mapped(const chem_mech* mech, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                          double rtol, double atol, double* h_inout, int32_t* status, const double* refs,
                          int32_t n_ref, double tol_T, double tol_Y, int32_t* zone, int64_t* n_mapped,
                          const chem_opts* opts, chem_stats* stats, void* stream);

/* Sensitivities (the discrete adjoint of the integrator).  The paper integrates forward only;
 * these entry points differentiate its solve: the map (phi_0, ln A) -> phi(dt) computed by the
 * accepted Rosenbrock steps of Sec. 2.3 (Eq. 2), with the step sizes frozen at the values the
 * controller chose.  A is the pre-exponential factor of the forward rate constant of each
 * reaction (of k_inf for fall-off reactions), in the file's reaction order.
 *
 * chem_integrate_record: chem_integrate in FP64 that also writes a checkpoint of every accepted
 * step: rec[(c * max_steps_rec + n) * (N + 1) + i] = phi_n[i] (the state the step starts from,
 * i < N) and [.. + N] = h_n (its size), N = K, for n < nsteps[c].  rec holds ncells *
 * max_steps_rec * (N + 1) doubles; a cell that needs more accepted steps ends with status
 * CHEM_CELL_RECORD_FULL.  opts->precision must be CHEM_PREC_FP64.  Device arrays only
 * (CHEM_EINVAL otherwise); status and nsteps must not be NULL. */
int chem_integrate_record(const chem_mech* mech, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                          double rtol, double atol, double* h_inout, int32_t* status, double* rec,
                          int32_t max_steps_rec, int32_t* nsteps, const chem_opts* opts, chem_stats* stats,
                          void* stream);

/* chem_adjoint: the reverse sweep over the checkpoints of chem_integrate_record (same mechanism
 * handle, pressure and ln A values).  Given gT[c] = dL/dT(dt) and gY[k * ncells + c] =
 * dL/dY_k(dt) of a scalar L of the final states (all K species; Y_K(dt) = 1 - sum of the others,
 * so its gradient enters as dL/dY_k - dL/dY_K), it writes
 *   gT0[c] = dL/dT(0), gY0[k * ncells + c] = dL/dY_k(0) for k < K-1 and 0 for k = K-1 (the
 *     solve never reads the input Y_K),
 *   g_lnA[r] = sum over cells of dL/d ln A_r (NULL: not computed), summed in a fixed order,
 *   g_lnA_cells[c * R + r] = the same per cell (NULL: not kept).
 * Per accepted step it recomputes the stages from the checkpoint, applies the transposed stage
 * solves with the same LU, the transposed Jacobians at the stage states, and the derivatives of
 * J and of f with respect to phi and ln A along the stage increments (dual numbers, exact up to
 * rounding).  A cell whose status is not CHEM_CELL_OK gets NaN gradients (and NaN in g_lnA).
 * Device arrays only; asynchronous on `stream`. */
int chem_adjoint(const chem_mech* mech, double p_Pa, int64_t ncells, const double* rec, int32_t max_steps_rec,
                 const int32_t* nsteps, const int32_t* status, const double* gT, const double* gY, double* gT0,
                 double* gY0, double* g_lnA, double* g_lnA_cells, void* stream);

/* ln A_r of every reaction (file order, R values, host arrays): read the mechanism's values, or
 * replace them (the device tables are updated synchronously; later calls use the new values). */
int chem_get_lnA(const chem_mech* mech, double* lnA);
int chem_set_lnA(chem_mech* mech, const double* lnA);

/* Per-cell counters of the last chem_integrate on this mechanism handle, copied to the
 * caller's arrays (device or host, ncells entries each, either may be NULL).  Valid until the
 * next chem_integrate on the handle. */
int chem_last_cell_counters(const chem_mech* mech, int32_t* steps, int32_t* rejects, int64_t ncells,
                            void* stream);

/* Diagnostic, not part of the chemistry: measures the FP64 fused-multiply-add throughput of the
 * current device (8 independent FMA chains per thread, 4 CTAs of 256 threads per SM, ~50 ms)
 * and returns it in TFLOP/s (2 flops per FMA).  It is the denominator of the roofline that the
 * benchmark reports for the integrate kernel, measured in the same process and clock state. */
int chem_probe_fp64_peak(double* tflops);

/* Diagnostic for the tests: y[i] = the exponential the rate kernels use (table-driven, Tang
 * 1989) of x[i], n entries, device arrays, asynchronous on `stream`. */
int chem_debug_exp(const double* x, double* y, int64_t n, void* stream);

/* Diagnostic for the tests: factors n dense N x N matrices (A: n x N x N, row-major, FP64,
 * 1 <= N <= 128) with the kernels' LU with partial pivoting (the dense LU of Sec. 2.3; ties go to
 * the lowest row) in the factor precision `precision` (CHEM_PREC_FP64: doubles, CHEM_PREC_MIXED:
 * floats, CHEM_PREC_MIXED_FF: FP32 pairs) in one of its three schedules, by one cell group of 2
 * warps per matrix: variant 0 column by column with four group barriers per column, 1 with two
 * (the pivot search of the next column fused into the trailing update; the integrate kernels'
 * default), 2 in panels of 8 columns.  All three give bitwise the same results.  Writes per matrix
 * the factors of P A = L D U' (N*N entries: the unit lower factor L's multipliers below the
 * diagonal, the pivots D on it, and above it the unit upper factor U' = D^-1 U, i.e. each row of
 * the upper factor U right of the diagonal times the reciprocal of its pivot, rounded once) to
 * `factors` and the reciprocal pivots (N entries) to `invdiag`, both
 * in the precision's storage (8 bytes per entry for doubles and pairs, 4 for floats), the row
 * permutation (N ints: row i of the factors is row perm[i] of the matrix) to `perm`, and 1 if a
 * pivot was exactly zero, else 0, to `singular` (n ints).  Device arrays, owned by the caller;
 * asynchronous on `stream`.  Returns CHEM_EINVAL for bad sizes, precision, variant or host
 * pointers. */
int chem_debug_lu(const double* A, int N, int64_t n, int precision, int variant, void* factors, void* invdiag,
                  int32_t* perm, int32_t* singular, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* chem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CHEMGPU_H */
