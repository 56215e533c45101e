// chemgpu kernels and C ABI (see include/chemgpu.h): the forward integrator, the one-shot
// rate and Jacobian kernels, and the host side (mechanism upload, launch shapes, CUDA graphs).
//
// GPU design (GB300, sm_103a).  A group of G warps integrates one cell at a time; a CTA holds
// several independent cell groups; a persistent grid pulls cells from a device work queue (one
// atomic per cell), so that cells of very different stiffness balance across SMs -- the
// on-device counterpart of the paper's MPI load balancing (Sec. 2.2).  Each group keeps its
// cell's whole working set in shared memory: the dense Jacobian (Sec. 2.3), the iteration
// matrix and its LU factors, the stage vectors and the per-reaction scratch.
//
// FP64 is the bottleneck on this part (measured ~0.5 T DFMA/s, 1/74 of FP32), and an FP64 warp
// instruction costs the same with 1 or 32 active lanes, so the work is laid out to keep all
// lanes busy: lanes stride over reactions, species and matrix entries, never over one scalar.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/chemgpu.h"
#include "adjoint.h"
#include "cell_device.cuh"
#include "chem_internal.h"

namespace {

// ------------------------------------------------------------------------------------------
// Optional per-phase cycle counters (compile with -DCHEM_PHASE_TIMERS): thread 0 of each cell
// group accumulates clock64() deltas per phase; read with chem_debug_phase_cycles().

#ifdef CHEM_PHASE_TIMERS
__device__ unsigned long long g_phase_cycles[8];
#define PHASE_BEGIN long long ph_t0_ = clock64();
#define PHASE_END(slot)                                                  \
  do {                                                                    \
    long long ph_t1_ = clock64();                                         \
    if (g.t == 0) atomicAdd(&g_phase_cycles[slot], (unsigned long long)(ph_t1_ - ph_t0_)); \
    ph_t0_ = ph_t1_;                                                      \
  } while (0)
#else
#define PHASE_BEGIN
#define PHASE_END(slot) \
  do {                  \
  } while (0)
#endif

// ------------------------------------------------------------------------------------------
// Kernels

// Threads per CTA of the integrate kernels (8 warps: with ~230 registers per thread that is the
// register file, and shared memory holds 4 cells of 53 species)
#ifndef CHEM_MAX_THREADS_PER_CTA
#define CHEM_MAX_THREADS_PER_CTA 256
#endif

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
};

// First-order forward-difference Jacobian (the alternative the paper measures the analytical
// Jacobian against, Sec. 2.3): N + 1 rate evaluations.  Column j = (f(y + d_j e_j) - f(y)) / d_j,
// d_j = 2^-26 max(|y_j|, s_j), s = 1 K for T and 1e-6 for the mass fractions (d_j taken as the
// step actually represented).  Leaves f(y) in w.f0 and -J in w.A (the analytical path's layout).
template <int G>
__device__ void cell_fd_jacobian(const DevMech& m, const Grp<G>& g, double p, const CellMem& w) {
  constexpr int NT = Grp<G>::NT;
  const int N = m.N;
  cell_rates(m, g, p, w.y, w.f0, eval_mem(w), (double*)nullptr, false);
  for (int j = 0; j < N; ++j) {
    const double yj = w.y[j];
    const double xj = yj + 0x1p-26 * fmax(fabs(yj), j == 0 ? 1.0 : 1e-6);
    const double dj = xj - yj;
    for (int i = g.t; i < N; i += NT) w.ynew[i] = (i == j) ? xj : w.y[i];
    g.sync();
    cell_rates(m, g, p, w.ynew, w.fs, eval_mem(w), (double*)nullptr, false);
    for (int i = g.t; i < N; i += NT) w.A[i * N + j] = -((w.fs[i] - w.f0[i]) / dj);
    g.sync();
  }
}

// ------------------------------------------------------------------------------------------
// Mixed precision (FP32 LU + FP64-residual iterative refinement).

// After an attempt whose FP32 refinement did not converge, the cell's next attempts use FP64
// factors directly (the iteration matrix changes slowly from step to step)
#ifndef CHEM_MIXED_FP64_RUN
#define CHEM_MIXED_FP64_RUN 16
#endif

// v 2^k for a power-of-two scaling whose result is at most 2 (an exponent-field add, no FP64
// operation); zero when v is zero or subnormal or the result would be subnormal.
__device__ inline double scale2(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0 || ef + k <= 0) return 0.0;
  return __longlong_as_double(b + ((long long)k << 52));
}

template <typename L>
__device__ inline L to_low(double v);
template <>
__device__ inline float to_low<float>(double v) { return __double2float_rn(v); }
template <>
__device__ inline FF to_low<FF>(double v) { return FF(v); }

// Equilibrate W = I gh - J by powers of two (row exponents er, then column exponents ec, from
// the largest entries) and factor S = D_r W D_c in the low precision L (FP32 or FP32 pairs) in
// buffer B; the reciprocal pivots go to invd.  The diagonal gh + (-J)_ii is formed once in FP64
// (in the residual vector, free until the stage solves), so the scans only compare exponents.
template <int G, typename L>
__device__ bool form_and_factor_low(const Grp<G>& g, const CellMem& w, int N, double gh, L* invd) {
  constexpr int NT = Grp<G>::NT;
  L* S = reinterpret_cast<L*>(w.B);
  double* dg = w.res;
  for (int i = g.t; i < N; i += NT) dg[i] = gh + w.A[i * N + i];
  g.sync();
  for (int i = g.t; i < N; i += NT) {
    int mx = 0;
    for (int j = 0; j < N; ++j) mx = max(mx, exp_field(i == j ? dg[i] : w.A[i * N + j]));
    w.er[i] = mx - 1023;
  }
  g.sync();
  for (int j = g.t; j < N; j += NT) {
    int mx = -2100;
    for (int i = 0; i < N; ++i) {
      const int ef = exp_field(i == j ? dg[j] : w.A[i * N + j]);
      if (ef > 0) mx = max(mx, ef - 1023 - w.er[i]);
    }
    w.ec[j] = (mx < -900) ? 0 : mx;
  }
  g.sync();
  for (int e = g.t; e < N * N; e += NT) {
    const int i = e / N, j = e - (e / N) * N;
    S[e] = to_low<L>(scale2(i == j ? dg[i] : w.A[e], -w.er[i] - w.ec[j]));
  }
  g.sync();
  return cell_lu<G, L>(g, S, N, w.piv, w.perm, invd);
}

// x <- W^-1 b through the low-precision factors of the equilibrated matrix S = D_r W D_c:
// z = D_r b, S v = z, x = D_c v (one warp).
template <typename L>
__device__ inline void low_solve(const CellMem& w, int N, const L* invd, const double* b, double* x) {
  warp_lu_solve_any<L>(reinterpret_cast<const L*>(w.B), N, w.perm, invd, w.er, w.ec, b, x);
}
__device__ inline const float* invd_of(const CellMem& w, float*) { return w.invd32; }
__device__ inline const FF* invd_of(const CellMem& w, FF*) { return reinterpret_cast<const FF*>(w.invdiag); }

// u <- W^-1 rhs with low-precision factors L: a solve, then up to refine_sweeps sweeps of
// r = rhs - W u (FP64, with the FP64 Jacobian), u += W_L^-1 r, until the last correction is
// below 1e-5 of the error-control scale atol + rtol |y|, or the residual of the sweep is at the
// rounding level of FP64 arithmetic (every |r_i| <= 2^-45 max_j |W_ij| max_j |u_j|, which
// covers the N <= 128 terms of a row; no further sweep can then improve u, which is as accurate
// as an FP64 solve can be checked to be).  Returns false if neither happens.  FP32 pairs with
// refine_sweeps = 0 take the first solve as it is.
template <int G, typename L>
__device__ bool stage_solve_low(const Grp<G>& g, const CellMem& w, const IntegrateArgs& a, int N, double gh,
                                double* u) {
  constexpr int NT = Grp<G>::NT;
  const L* invd = invd_of(w, (L*)nullptr);
  if (g.warp() == g.lead) low_solve<L>(w, N, invd, w.rhs, u);
  g.sync();
  if (a.refine_sweeps == 0) return true;
  double conv = INFINITY;
  for (int s = 0; s < a.refine_sweeps; ++s) {
    // residual r = rhs - W u = rhs - gh u + J u (the buffer holds -J); the exponent scan of u
    // and the row exponents er (|W_ij| < 2^(er_i + 1)) give the rounding level of each row
    bool above = false;
    for (int i = g.t; i < N; i += NT) {
      const double* Ji = w.A + (size_t)i * N;
      double s0 = 0.0, s1 = 0.0;
      int ue = 0;
      int j = 0;
      for (; j + 1 < N; j += 2) {
        s0 = fma(Ji[j], u[j], s0);
        s1 = fma(Ji[j + 1], u[j + 1], s1);
        ue = max(ue, max(exp_field(u[j]), exp_field(u[j + 1])));
      }
      if (j < N) {
        s0 = fma(Ji[j], u[j], s0);
        ue = max(ue, exp_field(u[j]));
      }
      const double r = fma(-gh, u[i], w.rhs[i]) - (s0 + s1);
      w.res[i] = r;
      // |r| < 2^(e_r - 1022) <= 2^-45 2^(er_i + 1) 2^(ue - 1022)  <=  e_r <= er_i + ue - 44
      above = above || exp_field(r) > w.er[i] + ue - 44;
    }
    g.sync();
    if (g.warp() == g.lead) low_solve<L>(w, N, invd, w.res, w.res);
    g.sync();
    double c = 0.0;
    for (int i = g.t; i < N; i += NT) {
      const double d = w.res[i];
      u[i] += d;
      c = Grp<G>::nanmax(c, fabs(d) / (a.atol + a.rtol * fabs(w.y[i])));
    }
    conv = g.max_nan_any(c, above);
    if (!above && conv == conv) conv = 0.0;  // residual at the FP64 rounding level
    if (conv <= 1e-5) break;
  }
  return conv <= 1e-5;
}

// u <- W^-1 rhs: FP64 factors (lowp 0: one solve), FP32 factors (1) or FP32 pairs (2).
template <int G>
__device__ bool stage_solve(const Grp<G>& g, const CellMem& w, const IntegrateArgs& a, int N, double gh, int lowp,
                            double* u) {
  constexpr int NT = Grp<G>::NT;
  if (lowp == 1) return stage_solve_low<G, float>(g, w, a, N, gh, u);
  if (lowp == 2) return stage_solve_low<G, FF>(g, w, a, N, gh, u);
  for (int i = g.t; i < N; i += NT) u[i] = w.rhs[i];
  g.sync();
  cell_solve(g, w.B, N, w.perm, w.invdiag, u);
  return true;
}

// Next cell of this group (an index into the arrays), or -1 when the launch's range is done.
template <int G>
__device__ inline int64_t next_cell(const IntegrateArgs& a, const Grp<G>& g, const CellMem& w, int64_t& static_next,
                                    int64_t stride) {
  int64_t c;
  if (a.use_queue) {
    if (g.t == 0) *w.slot = atomicAdd(a.queue, 1);
    g.sync();
    c = (int64_t)*w.slot;
    g.sync();
  } else {
    c = static_next;
    static_next += stride;
  }
  return c < a.count ? a.first + c : -1;
}

template <int G>
__global__ void __launch_bounds__(CHEM_MAX_THREADS_PER_CTA, 1) integrate_kernel(DevMech m, Plan plan, IntegrateArgs a) {
  extern __shared__ double smem[];
  Grp<G> g;
  g.init(threadIdx.x % Grp<G>::NT, threadIdx.x / Grp<G>::NT);
  CellMem w = carve(smem + (size_t)g.gid * plan.total, plan);
  g.red = w.red;
  constexpr int NT = Grp<G>::NT;
  const int N = m.N, K = m.K;
  const int groups_per_cta = blockDim.x / NT;
  const int64_t ngroups = (int64_t)gridDim.x * groups_per_cta;
  int64_t static_next = (int64_t)blockIdx.x * groups_per_cta + g.gid;
  const double gam = c_gamma;
  for (;;) {
    const int64_t cell = next_cell(a, g, w, static_next, ngroups);
    if (cell < 0) break;
    // load the state phi = [T, Y_1..Y_{K-1}]
    int bad = 0;
    for (int i = g.t; i < N; i += NT) {
      const double v = (i == 0) ? a.T[cell] : a.Y[(size_t)(i - 1) * a.ncells + cell];
      w.y[i] = v;
      bad |= !isfinite(v);
    }
    const double pc = a.p_cells ? 10.0 * a.p_cells[cell] : a.p;  // dyn/cm^2
    bad = (g.sum((double)bad) > 0.0) || !(a.T[cell] > 0.0) || !(pc > 0.0 && pc < INFINITY);
    int status = bad ? CHEM_CELL_BAD_INPUT : CHEM_CELL_OK;
    int nsteps = 0, nrej = 0;
    double h_next = 0.01 * a.dt;
    if (a.h_inout) {
      const double h0 = a.h_inout[cell];
      if (h0 > 0.0) h_next = fmin(h0, a.dt);
    }
    double t = 0.0, h = h_next;
    bool need_jac = true, last_rej = false;
    int f64_until = 0;
    g.sync();
    for (int attempt = 0; status == CHEM_CELL_OK; ++attempt) {
      if (attempt >= a.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
      if (h_next < 1e-14 * a.dt) { status = CHEM_CELL_H_UNDERFLOW; break; }
      PHASE_BEGIN
      if (need_jac) {
        if (a.fdjac) {
          cell_fd_jacobian(m, g, pc, w);
        } else {
          const CellScalars s0 = cell_rates(m, g, pc, w.y, w.f0, eval_mem(w), w.A, true);
          PHASE_END(0);
          cell_jacobian(m, g, s0, w.f0, eval_mem(w), w.A, w.B);
        }
        PHASE_END(1);
        need_jac = false;
      }
      // iteration matrix W = I/(gamma h) - J and its factors.  Mixed precision first tries the
      // FP32 factors of the equilibrated matrix with FP64-residual refinement; if a stage solve
      // does not converge the attempt is redone with FP64 factors.
      const double gh = 1.0 / (gam * h);
      const double invh = 1.0 / h;
      double err = INFINITY;
      // after a fallback the next attempts go straight to FP64 factors for a while
      for (int pass = (a.mixed && attempt >= f64_until) ? 0 : 1; pass < 2; ++pass) {
        const int lowp = pass == 0 ? a.mixed : 0;
        bool ok;
        if (lowp == 1) {
          ok = form_and_factor_low<G, float>(g, w, N, gh, w.invd32);
        } else if (lowp == 2) {
          ok = form_and_factor_low<G, FF>(g, w, N, gh, reinterpret_cast<FF*>(w.invdiag));
        } else {
          for (int e = g.t; e < N * N; e += NT) w.B[e] = w.A[e];
          g.sync();
          for (int i = g.t; i < N; i += NT) w.B[i * N + i] += gh;
          g.sync();
          ok = cell_lu<G, double>(g, w.B, N, w.piv, w.perm, w.invdiag);
        }
        PHASE_END(2);
        if (!ok) break;  // exactly singular: reject the attempt
        bool conv = true;
        // stage 1
        for (int i = g.t; i < N; i += NT) w.rhs[i] = w.f0[i];
        g.sync();
        conv = stage_solve(g, w, a, N, gh, lowp, w.u[0]);
        PHASE_END(3);
        // stage 2
        if (conv) {
          for (int i = g.t; i < N; i += NT) w.ynew[i] = fma(c_a21, w.u[0][i], w.y[i]);
          g.sync();
          cell_rates(m, g, pc, w.ynew, w.fs, eval_mem(w), (double*)nullptr, false);
          PHASE_END(4);
          for (int i = g.t; i < N; i += NT) w.rhs[i] = fma(c_c21 * invh, w.u[0][i], w.fs[i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, lowp, w.u[1]);
          PHASE_END(3);
        }
        // stage 3
        if (conv) {
          for (int i = g.t; i < N; i += NT) w.ynew[i] = w.y[i] + c_a31 * w.u[0][i] + c_a32 * w.u[1][i];
          g.sync();
          cell_rates(m, g, pc, w.ynew, w.fs, eval_mem(w), (double*)nullptr, false);
          PHASE_END(4);
          for (int i = g.t; i < N; i += NT)
            w.rhs[i] = w.fs[i] + invh * (c_c31 * w.u[0][i] + c_c32 * w.u[1][i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, lowp, w.u[2]);
        }
        // stage 4 (same argument as stage 3)
        if (conv) {
          for (int i = g.t; i < N; i += NT)
            w.rhs[i] = w.fs[i] + invh * (c_c41 * w.u[0][i] + c_c42 * w.u[1][i] + c_c43 * w.u[2][i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, lowp, w.u[3]);
        }
        if (!conv) {
          if (g.t == 0) atomicAdd(&a.totals[3], 1ull);
          f64_until = attempt + CHEM_MIXED_FP64_RUN;
          continue;  // redo this attempt with FP64 factors
        }
        // solution, embedded error, filtered through (I - gamma h J)^-1 = W^-1 / (gamma h)
        // (the filter only feeds the step-size control, so FP32 factors need no refinement)
        for (int i = g.t; i < N; i += NT) {
          w.ynew[i] = w.y[i] + c_m[0] * w.u[0][i] + c_m[1] * w.u[1][i] + c_m[2] * w.u[2][i] + c_m[3] * w.u[3][i];
          w.rhs[i] = c_e[0] * w.u[0][i] + c_e[1] * w.u[1][i] + c_e[2] * w.u[2][i] + c_e[3] * w.u[3][i];
        }
        g.sync();
        if (lowp == 1) {
          if (g.warp() == g.lead) low_solve<float>(w, N, w.invd32, w.rhs, w.err);
          g.sync();
        } else if (lowp == 2) {
          if (g.warp() == g.lead) low_solve<FF>(w, N, reinterpret_cast<const FF*>(w.invdiag), w.rhs, w.err);
          g.sync();
        } else {
          for (int i = g.t; i < N; i += NT) w.err[i] = w.rhs[i];
          g.sync();
          cell_solve(g, w.B, N, w.perm, w.invdiag, w.err);
        }
        PHASE_END(3);
        double e = 0.0;
        for (int i = g.t; i < N; i += NT) {
          const double sc = a.atol + a.rtol * fmax(fabs(w.y[i]), fabs(w.ynew[i]));
          e = Grp<G>::nanmax(e, fabs(w.err[i] * gh) / sc);
        }
        err = g.max_nan(e);
        break;
      }
      double fac;
      if (err <= 1.0) {
        if (a.rec) {
          // checkpoint (phi_n, h_n) of the accepted step for the adjoint
          if (nsteps >= a.rec_cap) { status = CHEM_CELL_RECORD_FULL; break; }
          double* ck = a.rec + ((size_t)cell * a.rec_cap + nsteps) * (N + 1);
          for (int i = g.t; i < N; i += NT) ck[i] = w.y[i];
          if (g.t == 0) ck[N] = h;
        }
        t = (h >= a.dt - t) ? a.dt : t + h;
        for (int i = g.t; i < N; i += NT) w.y[i] = w.ynew[i];
        g.sync();
        ++nsteps;
        need_jac = true;
        fac = fmin(6.0, fmax(0.2, 0.9 * pow(err, -0.25)));
        if (last_rej) fac = fmin(fac, 1.0);
        last_rej = false;
        h_next = h * fac;
        if (t >= a.dt) break;
      } else {
        ++nrej;
        fac = (err == err && err < INFINITY) ? fmax(0.2, 0.9 * pow(err, -0.25)) : 0.2;
        fac = fmin(fac, 1.0);
        last_rej = true;
        h_next = h * fac;
      }
      h = fmin(h_next, a.dt - t);
      PHASE_END(5);
    }
    // store phi and Y_K = 1 - sum
    double ysum = 0.0;
    for (int i = g.t; i < N; i += NT) {
      const double v = w.y[i];
      if (i == 0) a.T[cell] = v;
      else { a.Y[(size_t)(i - 1) * a.ncells + cell] = v; ysum += v; }
    }
    ysum = g.sum(ysum);
    if (g.t == 0) {
      if (status != CHEM_CELL_BAD_INPUT) a.Y[(size_t)(K - 1) * a.ncells + cell] = 1.0 - ysum;
      if (a.h_inout && status != CHEM_CELL_BAD_INPUT) a.h_inout[cell] = h_next;
      if (a.status) a.status[cell] = status;
      if (a.steps_out) a.steps_out[cell] = nsteps;
      if (a.rej_out) a.rej_out[cell] = nrej;
      atomicAdd(&a.totals[0], (unsigned long long)nsteps);
      atomicAdd(&a.totals[1], (unsigned long long)nrej);
      if (status != CHEM_CELL_OK) atomicAdd(&a.totals[2], 1ull);
    }
    g.sync();
  }
}

// ------------------------------------------------------------------------------------------
// Seulex (the paper's integrator, Sec. 2.3; Hairer & Wanner IV.9): the linearly implicit Euler
// method with extrapolation.  Per macro step H from y with J = J(y): column j takes n_j = j
// sub-steps of h = H/j, (I/h - J) d = f(y_i), y_{i+1} = y_i + d (one LU of I/h - J per column),
// T_{j,1} = y_{n_j}; Aitken-Neville T_{j,l} = T_{j,l-1} + (T_{j,l-1} - T_{j-1,l-1}) /
// (n_j/n_{j-l+1} - 1); err_j = max norm of T_{j,j} - T_{j,j-1} (scale atol + rtol max(|y|,
// |T_jj|)), fac_j = min(4, max(0.02, 0.94 err_j^(-1/j))).  Target column k in [2, kmax-1]:
// accept at column k-1 or k if err <= 1, give up at k if err > (n_{k+1}/n_1)^2, decide at k+1.
// The next target and step minimise the work per unit step A_j / (H fac_j), A_j the cost of
// columns 1..j in rate-evaluation units (Jacobian 2.5, LU 2, rate evaluation 1, solve 0.2).  A
// give-up keeps J and shrinks H by min(fac, 1/2); a singular matrix or a non-finite error by 1/5.
// The tableau row lives in eight of the cell's vectors and is updated element by element.
constexpr int kSeulexKmax = 8;

__device__ inline double seulex_work(int j) {
  // A_1 = 2.5 + 2 + (0.2 + 1); A_j = A_{j-1} + 2 + 0.2 j + (j - 1)
  double a = 2.5 + 2.0 + 1.2;
  for (int i = 2; i <= j; ++i) a += 2.0 + 0.2 * i + (i - 1);
  return a;
}

template <int G>
__global__ void __launch_bounds__(CHEM_MAX_THREADS_PER_CTA, 1) seulex_kernel(DevMech m, Plan plan, IntegrateArgs a) {
  extern __shared__ double smem[];
  Grp<G> g;
  g.init(threadIdx.x % Grp<G>::NT, threadIdx.x / Grp<G>::NT);
  CellMem w = carve(smem + (size_t)g.gid * plan.total, plan);
  g.red = w.red;
  constexpr int NT = Grp<G>::NT;
  constexpr int kmax = kSeulexKmax;
  const int N = m.N, K = m.K;
  const int groups_per_cta = blockDim.x / NT;
  const int64_t ngroups = (int64_t)gridDim.x * groups_per_cta;
  int64_t static_next = (int64_t)blockIdx.x * groups_per_cta + g.gid;
  // tableau row T_1..T_8 in the vectors u0..u3, err, res and the two last ones (vector slots
  // 4..8 and 11..13 of the plan), addressed arithmetically so that nothing goes to local memory
  const int n2 = (int)(w.ynew - w.y);
  auto tab = [&](int l) { return w.y + (size_t)(l + 3 + (l >= 6 ? 2 : 0)) * n2; };
  double* yi = w.ynew;
  double* fi = w.fs;
  double* d = w.rhs;
  for (;;) {
    const int64_t cell = next_cell(a, g, w, static_next, ngroups);
    if (cell < 0) break;
    int bad = 0;
    for (int i = g.t; i < N; i += NT) {
      const double v = (i == 0) ? a.T[cell] : a.Y[(size_t)(i - 1) * a.ncells + cell];
      w.y[i] = v;
      bad |= !isfinite(v);
    }
    const double pc = a.p_cells ? 10.0 * a.p_cells[cell] : a.p;  // dyn/cm^2
    bad = (g.sum((double)bad) > 0.0) || !(a.T[cell] > 0.0) || !(pc > 0.0 && pc < INFINITY);
    int status = bad ? CHEM_CELL_BAD_INPUT : CHEM_CELL_OK;
    int nsteps = 0, nrej = 0;
    double H_next = 0.01 * a.dt;
    if (a.h_inout) {
      const double h0 = a.h_inout[cell];
      if (h0 > 0.0) H_next = fmin(h0, a.dt);
    }
    double t = 0.0, H = H_next;
    int k = 2;
    bool need_jac = true, last_rej = false;
    g.sync();
    for (int attempt = 0; status == CHEM_CELL_OK; ++attempt) {
      if (attempt >= a.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
      if (H_next < 1e-14 * a.dt) { status = CHEM_CELL_H_UNDERFLOW; break; }
      if (need_jac) {
        const CellScalars s0 = cell_rates(m, g, pc, w.y, w.f0, eval_mem(w), w.A, true);
        cell_jacobian(m, g, s0, w.f0, eval_mem(w), w.A, w.B);
        need_jac = false;
      }
      double fac_cur = 0.2, fac_prv = 0.2;  // fac of the last column computed and of the one before
      int accepted = 0, last = 0;
      bool badstep = false;
      for (int j = 1; j <= k + 1; ++j) {
        last = j;
        const double gh = (double)j / H;  // 1/h
        for (int e = g.t; e < N * N; e += NT) w.B[e] = w.A[e];
        g.sync();
        for (int i = g.t; i < N; i += NT) w.B[i * N + i] += gh;
        g.sync();
        if (!cell_lu<G, double>(g, w.B, N, w.piv, w.perm, w.invdiag)) { badstep = true; break; }
        for (int i = g.t; i < N; i += NT) yi[i] = w.y[i];
        for (int sub = 0; sub < j; ++sub) {
          const double* fsrc = w.f0;
          if (sub > 0) {
            g.sync();
            cell_rates(m, g, pc, yi, fi, eval_mem(w), (double*)nullptr, false);
            fsrc = fi;
          }
          for (int i = g.t; i < N; i += NT) d[i] = fsrc[i];
          g.sync();
          cell_solve(g, w.B, N, w.perm, w.invdiag, d);
          for (int i = g.t; i < N; i += NT) yi[i] += d[i];
        }
        // extrapolation, element by element, and the error of column j
        double e = 0.0;
        for (int i = g.t; i < N; i += NT) {
          double q = yi[i];
          for (int l = 2; l <= j; ++l) {
            const double r = (double)j / (double)(j - l + 1);
            double* tl = tab(l - 1);
            const double qn = q + (q - tl[i]) / (r - 1.0);
            tl[i] = q;
            q = qn;
          }
          tab(j)[i] = q;
          if (j >= 2) {
            const double sc = a.atol + a.rtol * fmax(fabs(w.y[i]), fabs(q));
            e = Grp<G>::nanmax(e, fabs(q - tab(j - 1)[i]) / sc);
          }
        }
        g.sync();
        if (j < 2) continue;
        e = g.max_nan(e);
        if (!(e < INFINITY)) { badstep = true; break; }  // NaN or infinite
        fac_prv = fac_cur;
        fac_cur = (e > 0.0) ? fmin(4.0, fmax(0.02, 0.94 * pow(e, -1.0 / j))) : 4.0;
        if (j == k - 1) {
          if (e <= 1.0) { accepted = j; break; }
        } else if (j == k) {
          if (e <= 1.0) { accepted = j; break; }
          const double ratio = (double)(k + 1);  // n_{k+1} / n_1
          if (e > ratio * ratio) break;
        } else if (j == k + 1) {
          if (e <= 1.0) accepted = j;
          break;
        }
      }
      if (accepted) {
        const int c = accepted;
        t = (H >= a.dt - t) ? a.dt : t + H;
        const double* tc = tab(c);
        for (int i = g.t; i < N; i += NT) w.y[i] = tc[i];
        g.sync();
        ++nsteps;
        need_jac = true;
        // fac_cur = fac_c, fac_prv = fac_{c-1} (c is the last column computed)
        int knew;
        double Hn;
        if (c == 2) {
          knew = 3;
          Hn = H * fac_cur * (last_rej ? 1.0 : seulex_work(3) / seulex_work(2));
        } else if (c <= k) {
          const double wc = seulex_work(c) / (H * fac_cur), wc1 = seulex_work(c - 1) / (H * fac_prv);
          knew = c;
          if (wc1 < 0.8 * wc) knew = c - 1;
          else if (c == k && wc < 0.9 * wc1) knew = c + 1;
          Hn = H * (knew < c ? fac_prv : fac_cur) * (knew > c ? seulex_work(knew) / seulex_work(c) : 1.0);
        } else {
          const double wc = seulex_work(c) / (H * fac_cur), wc1 = seulex_work(c - 1) / (H * fac_prv);
          knew = c - 1;
          if (wc < 0.9 * wc1) knew = c;
          Hn = H * (knew == c ? fac_cur : fac_prv);
        }
        if (last_rej) { Hn = fmin(Hn, H); knew = min(knew, c); }
        k = max(2, min(knew, kmax - 1));
        last_rej = false;
        H_next = Hn;
        if (t >= a.dt) break;
      } else {
        ++nrej;
        last_rej = true;
        if (badstep) {
          H_next = H * 0.2;
        } else {
          // gave up at column k (fac_k = fac_cur) or k+1 (fac_k = fac_prv)
          const int mc = min(k, last);
          H_next = H * fmin(last == k ? fac_cur : fac_prv, 0.5);
          k = max(2, mc);
        }
      }
      H = fmin(H_next, a.dt - t);
    }
    double ysum = 0.0;
    for (int i = g.t; i < N; i += NT) {
      const double v = w.y[i];
      if (i == 0) a.T[cell] = v;
      else { a.Y[(size_t)(i - 1) * a.ncells + cell] = v; ysum += v; }
    }
    ysum = g.sum(ysum);
    if (g.t == 0) {
      if (status != CHEM_CELL_BAD_INPUT) a.Y[(size_t)(K - 1) * a.ncells + cell] = 1.0 - ysum;
      if (a.h_inout && status != CHEM_CELL_BAD_INPUT) a.h_inout[cell] = H_next;
      if (a.status) a.status[cell] = status;
      if (a.steps_out) a.steps_out[cell] = nsteps;
      if (a.rej_out) a.rej_out[cell] = nrej;
      atomicAdd(&a.totals[0], (unsigned long long)nsteps);
      atomicAdd(&a.totals[1], (unsigned long long)nrej);
      if (status != CHEM_CELL_OK) atomicAdd(&a.totals[2], 1ull);
    }
    g.sync();
  }
}

// One-shot source term / Jacobian for chem_rates and chem_jacobian.
template <int G>
__global__ void __launch_bounds__(256, 1) rates_kernel(DevMech m, Plan plan, double p, const double* T, const double* Y,
                                                    int64_t ncells, double* out_f, double* out_J) {
  extern __shared__ double smem[];
  Grp<G> g;
  g.init(threadIdx.x % Grp<G>::NT, threadIdx.x / Grp<G>::NT);
  CellMem w = carve(smem + (size_t)g.gid * plan.total, plan);
  g.red = w.red;
  constexpr int NT = Grp<G>::NT;
  const int N = m.N;
  const int groups_per_cta = blockDim.x / NT;
  const int64_t ngroups = (int64_t)gridDim.x * groups_per_cta;
  for (int64_t cell = (int64_t)blockIdx.x * groups_per_cta + g.gid; cell < ncells; cell += ngroups) {
    for (int i = g.t; i < N; i += NT) w.y[i] = (i == 0) ? T[cell] : Y[(size_t)(i - 1) * ncells + cell];
    g.sync();
    const bool jac = out_J != nullptr;
    CellScalars s = cell_rates(m, g, p, w.y, w.f0, eval_mem(w), w.A, jac);
    if (jac) {
      cell_jacobian(m, g, s, w.f0, eval_mem(w), w.A, w.B);
      double* o = out_J + (size_t)cell * N * N;
      for (int e = g.t; e < N * N; e += NT) o[e] = -w.A[e];
    }
    if (out_f)
      for (int i = g.t; i < N; i += NT) out_f[(size_t)i * ncells + cell] = w.f0[i];
    g.sync();
  }
}

// Diagnostic: FP64 FMA pipe throughput (8 independent chains per thread).
__global__ void __launch_bounds__(256) fp64_peak_kernel(double* out, int iters, double s) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
         a7 = a0 + 7;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, s, 0.5); a1 = fma(a1, s, 0.5); a2 = fma(a2, s, 0.5); a3 = fma(a3, s, 0.5);
    a4 = fma(a4, s, 0.5); a5 = fma(a5, s, 0.5); a6 = fma(a6, s, 0.5); a7 = fma(a7, s, 0.5);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// ------------------------------------------------------------------------------------------
// Zonal reference-cell mapping (DLBFoam's, Sec. 2.2): cells whose state lies within a tolerance
// of a reference state (an ambient zone of low reactivity) are not solved; they receive the
// reference state's change over dt.  Three small kernels around the ordinary solve: classify
// (and compact the cells to solve), gather (the compact state, plus the references appended),
// scatter (solved cells back, mapped cells shifted by their reference's change).

// refs: [n_ref][1 + K] = T, Y_0 .. Y_{K-1}.  zone[c] = first reference within |T - T_r| <= tol_T
// and max_k |Y_k - Y_r,k| <= tol_Y, or -1; cells with zone -1 get a compact position pos[c].
__global__ void map_classify_kernel(const double* T, const double* Y, int64_t ncells, int K, const double* refs,
                                    int n_ref, double tol_T, double tol_Y, int32_t* zone, int64_t* pos,
                                    int64_t* list, unsigned long long* count) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int z = -1;
  for (int r = 0; r < n_ref && z < 0; ++r) {
    const double* rf = refs + (size_t)r * (1 + K);
    bool ok = fabs(T[c] - rf[0]) <= tol_T;
    for (int k = 0; ok && k < K; ++k) ok = fabs(Y[(size_t)k * ncells + c] - rf[1 + k]) <= tol_Y;
    if (ok) z = r;
  }
  zone[c] = z;
  if (z < 0) {
    const int64_t i = (int64_t)atomicAdd(count, 1ull);
    pos[c] = i;
    list[i] = c;
  }
}

// compact state: the n_un cells to solve, then the n_ref references (cold start)
__global__ void map_gather_kernel(const double* T, const double* Y, const double* h, int64_t ncells, int K,
                                  const double* refs, int n_ref, const int64_t* list, int64_t n_un, double* Tc,
                                  double* Yc, double* hc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = n_un + n_ref;
  if (i >= nc) return;
  if (i < n_un) {
    const int64_t c = list[i];
    Tc[i] = T[c];
    for (int k = 0; k < K; ++k) Yc[(size_t)k * nc + i] = Y[(size_t)k * ncells + c];
    hc[i] = h ? h[c] : 0.0;
  } else {
    const double* rf = refs + (size_t)(i - n_un) * (1 + K);
    Tc[i] = rf[0];
    for (int k = 0; k < K; ++k) Yc[(size_t)k * nc + i] = rf[1 + k];
    hc[i] = 0.0;
  }
}

__global__ void map_scatter_kernel(double* T, double* Y, double* h, int32_t* status, int64_t ncells, int K,
                                   const double* refs, const int32_t* zone, const int64_t* pos, int64_t n_un,
                                   int n_ref, const double* Tc, const double* Yc, const double* hc,
                                   const int32_t* sc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const int64_t nc = n_un + n_ref;
  const int z = zone[c];
  if (z < 0) {
    const int64_t i = pos[c];
    T[c] = Tc[i];
    for (int k = 0; k < K; ++k) Y[(size_t)k * ncells + c] = Yc[(size_t)k * nc + i];
    if (h) h[c] = hc[i];
    if (status) status[c] = sc[i];
  } else {
    const int64_t i = n_un + z;
    const double* rf = refs + (size_t)z * (1 + K);
    T[c] += Tc[i] - rf[0];
    double ysum = 0.0;
    for (int k = 0; k < K - 1; ++k) {
      const double v = Y[(size_t)k * ncells + c] + (Yc[(size_t)k * nc + i] - rf[1 + k]);
      Y[(size_t)k * ncells + c] = v;
      ysum += v;
    }
    Y[(size_t)(K - 1) * ncells + c] = 1.0 - ysum;
    if (status) status[c] = sc[i];
  }
}

// ------------------------------------------------------------------------------------------
// Scratch of chem_integrate_noalloc: a fixed device array instead of library allocations.
// Layout: [0, 4) work-queue counter, [64, 96) the four call totals, [256, ...) per-cell accepted
// step counts, then per-cell rejection counts, for at most kNoAllocMaxCells cells (2 MiB).
constexpr int64_t kNoAllocMaxCells = 262144;
constexpr size_t kNoAllocCounters = 256;
constexpr size_t kNoAllocScratchBytes = kNoAllocCounters + 2 * sizeof(int32_t) * (size_t)kNoAllocMaxCells;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

__global__ void exp_probe_kernel(const double* x, double* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_fast(x[i]);
}

}  // namespace

// ==========================================================================================
// Host side

struct GraphKey {
  IntegrateArgs a;
  chem_opts o;
};
struct GraphCache {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
};

struct chem_mech {
  HostMech host;
  DevMech dev;
  GraphCache graph;
  void* dbuf = nullptr;
  int device = 0;
  int num_sms = 0;
  size_t max_smem = 0;
  // workspaces (grow-only)
  unsigned long long* d_totals = nullptr;
  int* d_queue = nullptr;
  int32_t* d_steps = nullptr;
  int32_t* d_rej = nullptr;
  int64_t cap_cells = 0;
  void* d_stage = nullptr;  // device staging for host-pointer calls
  size_t cap_stage = 0;
  void* d_map_ws = nullptr;  // reference-mapping workspace
  size_t cap_map_ws = 0;
  double* d_adj_ws = nullptr;  // reverse-sweep workspace
  size_t cap_adj_ws = 0;
  int* d_adj_counters = nullptr;
};

namespace {

thread_local std::string g_err;

int set_err(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return set_err(CHEM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int ensure_cells(chem_mech* m, int64_t ncells) {
  if (ncells <= m->cap_cells) return 0;
  cudaFree(m->d_steps);
  cudaFree(m->d_rej);
  m->d_steps = m->d_rej = nullptr;
  m->cap_cells = 0;
  CK(cudaMalloc(&m->d_steps, sizeof(int32_t) * ncells));
  CK(cudaMalloc(&m->d_rej, sizeof(int32_t) * ncells));
  m->cap_cells = ncells;
  return 0;
}

int ensure_stage(chem_mech* m, size_t bytes) {
  if (bytes <= m->cap_stage) return 0;
  cudaFree(m->d_stage);
  m->d_stage = nullptr;
  m->cap_stage = 0;
  CK(cudaMalloc(&m->d_stage, bytes));
  m->cap_stage = bytes;
  return 0;
}

struct Launch {
  int G, cells_per_cta, grid, threads;
  size_t smem;
  Plan plan;
};

const void* integrate_fn(int G, int solver) {
  if (solver == CHEM_SOLVER_SEULEX)
    return G == 1 ? (const void*)seulex_kernel<1>
           : G == 2 ? (const void*)seulex_kernel<2>
           : G == 4 ? (const void*)seulex_kernel<4>
                    : (const void*)seulex_kernel<8>;
  return G == 1 ? (const void*)integrate_kernel<1>
         : G == 2 ? (const void*)integrate_kernel<2>
         : G == 4 ? (const void*)integrate_kernel<4>
                  : (const void*)integrate_kernel<8>;
}
const void* rates_fn(int G) {
  return G == 1 ? (const void*)rates_kernel<1>
         : G == 2 ? (const void*)rates_kernel<2>
         : G == 4 ? (const void*)rates_kernel<4>
                  : (const void*)rates_kernel<8>;
}

void launch_integrate(const Launch& L, cudaStream_t st, const DevMech& d, const IntegrateArgs& a) {
  if (a.solver == CHEM_SOLVER_SEULEX) {
    switch (L.G) {
      case 1: seulex_kernel<1><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
      case 2: seulex_kernel<2><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
      case 4: seulex_kernel<4><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
      default: seulex_kernel<8><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
    }
    return;
  }
  switch (L.G) {
    case 1: integrate_kernel<1><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
    case 2: integrate_kernel<2><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
    case 4: integrate_kernel<4><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
    default: integrate_kernel<8><<<L.grid, L.threads, L.smem, st>>>(d, L.plan, a); break;
  }
}

// Launch shape: G warps per cell, as many cells per CTA as the shared memory allows (at most 8
// warps per CTA, 15 named barriers), one persistent CTA wave.
int pick_launch(const chem_mech* m, int64_t ncells, int want_G, int want_cpc, int want_ctas_per_sm, bool integ,
                Launch& L, int solver = CHEM_SOLVER_ROSENBROCK) {
  int G = want_G;
  if (G <= 0) {
    // automatic: about 8 warps per SM -- G = 8 / (cells that fit), a power of two in 1..8, and
    // at least 2 warps per cell from 32 species up
    const size_t per_cell2 = (size_t)make_plan(m->host.K, m->host.R, m->dev.n_pd, 2).total * sizeof(double);
    const int fit = (int)std::max<size_t>(1, m->max_smem / per_cell2);
    G = 1;
    while (G < 8 && G * fit < 8) G *= 2;
    if (m->host.K >= 32 && G < 2) G = 2;
    if (m->host.K < 32 && fit >= 8) G = 1;
  }
  if (G != 1 && G != 2 && G != 4 && G != 8) return set_err(CHEM_EINVAL, "warps_per_cell must be 1, 2, 4 or 8");
  L.G = G;
  L.plan = make_plan(m->host.K, m->host.R, m->dev.n_pd, G);
  const size_t per_cell = (size_t)L.plan.total * sizeof(double);
  int max_cpc = (int)std::min<size_t>(std::max(1, std::min(CHEM_MAX_THREADS_PER_CTA / 32 / G, 15)),
                                      m->max_smem / per_cell);
  if (max_cpc < 1)
    return set_err(CHEM_ESIZE, "mechanism working set (" + std::to_string(per_cell) +
                                   " B per cell) exceeds the shared memory of one CTA");
  const int cpc = want_cpc > 0 ? std::min(want_cpc, max_cpc) : max_cpc;
  L.cells_per_cta = cpc;
  L.threads = 32 * G * cpc;
  L.smem = per_cell * cpc;
  const void* kernel = integ ? integrate_fn(G, solver) : rates_fn(G);
  int occ = 0;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, L.threads, L.smem));
  if (occ < 1) return set_err(CHEM_ESIZE, "kernel cannot be resident with the requested shared memory");
  const int cps = want_ctas_per_sm > 0 ? std::min(want_ctas_per_sm, occ) : occ;
  const int64_t need = (ncells + cpc - 1) / cpc;
  L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)m->num_sms * cps));
  return 0;
}

// Enqueue one integrate call on `st`: reset the totals, then for each batch (all cells in one
// batch unless batch_cells > 0) reset the queue and launch.
int enqueue_integrate(chem_mech* m, const chem_opts& o, IntegrateArgs a, cudaStream_t st) {
  CK(cudaMemsetAsync(a.totals, 0, 4 * sizeof(unsigned long long), st));
  const int64_t total = a.count;
  const int64_t batch = o.batch_cells > 0 ? (int64_t)o.batch_cells : total;
  for (int64_t first = 0; first < total; first += batch) {
    a.first = first;
    a.count = std::min(batch, total - first);
    Launch L;
    int rc = pick_launch(m, a.count, o.warps_per_cell, o.cells_per_cta, o.ctas_per_sm, true, L, a.solver);
    if (rc) return rc;
    CK(cudaMemsetAsync(a.queue, 0, sizeof(int), st));
    launch_integrate(L, st, m->dev, a);
    CK(cudaGetLastError());
  }
  return 0;
}

// CUDA-graph launch: the library records enqueue_integrate on its own stream once per argument
// set (stream capture), instantiates it, and replays it on the caller's stream.
int launch_via_graph(chem_mech* m, const chem_opts& o, const IntegrateArgs& a, cudaStream_t st) {
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.a = a;
  key.o = o;
  GraphCache& gc = m->graph;
  if (!gc.exec || std::memcmp(&gc.key, &key, sizeof(key)) != 0) {
    if (gc.exec) { cudaGraphExecDestroy(gc.exec); gc.exec = nullptr; }
    if (!gc.capture_stream) CK(cudaStreamCreateWithFlags(&gc.capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(gc.capture_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_integrate(m, o, a, gc.capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(gc.capture_stream, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return set_err(CHEM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { gc.exec = nullptr; return set_err(CHEM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
    gc.key = key;
  }
  CK(cudaGraphLaunch(gc.exec, st));
  return 0;
}

}  // namespace

extern "C" {

const char* chem_last_error(void) { return g_err.c_str(); }

void chem_default_opts(chem_opts* o) {
  if (!o) return;
  o->precision = CHEM_PREC_FP64;
  o->refine_sweeps = 2;
  o->max_steps = 100000;
  o->use_queue = 1;
  o->cells_per_cta = 0;
  o->ctas_per_sm = 0;
  o->warps_per_cell = 0;
  o->use_graph = 0;
  o->batch_cells = 0;
  o->solver = CHEM_SOLVER_ROSENBROCK;
  o->jacobian = CHEM_JAC_ANALYTIC;
}

// The tables of a parsed mechanism in file order, as text (see chem_describe_mechanism).
static std::string describe_tables(const HostMech& h) {
  std::string s;
  char num[40];
  auto put = [&](double v) {
    snprintf(num, sizeof num, " %.17g", v);
    s += num;
  };
  s += "species " + std::to_string(h.K) + "\n";
  for (int k = 0; k < h.K; ++k) {
    const double* sp = &h.sp[(size_t)k * kSpDoubles];
    s += "sp";
    put(sp[0]);
    for (int i = 2; i < kSpDoubles; ++i) put(sp[i]);  // Tmid, low a1..a7, high a1..a7
    s += "\n";
  }
  s += "reactions " + std::to_string(h.R) + "\n";
  std::vector<int> dev_of(h.R);
  for (int dr = 0; dr < h.R; ++dr) dev_of[h.order[dr]] = dr;
  for (int r = 0; r < h.R; ++r) {
    const int dr = dev_of[r];
    const int* ii = &h.rxi[(size_t)dr * kRxInts];
    const double* d = &h.rxd[(size_t)dr * kRxDoubles];
    const double* q = dr < h.n_fo ? &h.fo[(size_t)dr * kFoDoubles] : nullptr;
    const int type = q ? (q[7] != 0.0 ? kTroe : kLindemann) : (dr < h.n_fo + h.n_tb ? kThirdBody : kElementary);
    s += "rx " + std::to_string(type);
    for (int side = 0; side < 2; ++side) {
      int a = ii[2 * side], b = ii[2 * side + 1];
      if (a > b) std::swap(a, b);
      s += " " + std::to_string((a >= 0) + (b >= 0));
      if (a >= 0) s += " " + std::to_string(a);
      if (b >= 0) s += " " + std::to_string(b);
    }
    put(std::exp(d[0]));
    put(d[1]);
    put(d[2]);
    if (type >= kThirdBody) {
      s += " eff";
      for (int k = 0; k < h.K; ++k) put(h.eff[(size_t)dr * h.K + k]);
    }
    if (q) {
      s += " low";
      put(std::exp(q[0]));
      put(q[1]);
      put(q[2]);
      if (type == kTroe) {
        s += " troe";
        for (int i = 3; i < 7; ++i) put(q[i]);
      }
    }
    s += "\n";
  }
  return s;
}

int chem_describe_mechanism(const char* path, char* buf, int64_t cap, int64_t* need) {
  if (!path || !need || (cap > 0 && !buf)) return set_err(CHEM_EINVAL, "chem_describe_mechanism: NULL argument");
  HostMech h;
  std::string err;
  if (!parse_mechanism(path, h, err)) return set_err(CHEM_EFILE, err);
  const std::string s = describe_tables(h);
  *need = (int64_t)s.size() + 1;
  if (cap <= 0) return CHEM_OK;
  if (cap < *need) return set_err(CHEM_ESIZE, "chem_describe_mechanism: buffer too small");
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return CHEM_OK;
}

int chem_load_mechanism(const char* path, chem_mech** out) {
  if (!path || !out) return set_err(CHEM_EINVAL, "chem_load_mechanism: NULL argument");
  *out = nullptr;
  chem_mech* m = new chem_mech();
  std::string err;
  if (!parse_mechanism(path, m->host, err)) {
    delete m;
    return set_err(CHEM_EFILE, err);
  }
  const HostMech& h = m->host;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  int smem_optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
  if (e != cudaSuccess) {
    delete m;
    return set_err(CHEM_ECUDA, std::string("chem_load_mechanism: ") + cudaGetErrorString(e));
  }
  m->max_smem = (size_t)smem_optin;
  // one device allocation for all tables, each 256-byte aligned
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_sp = place(h.sp.size() * sizeof(double));
  const size_t o_rxd = place(h.rxd.size() * sizeof(double));
  const size_t o_rxi = place(h.rxi.size() * sizeof(int));
  const size_t o_dnu = place(h.dnu.size() * sizeof(int));
  const size_t o_eff = place(std::max<size_t>(1, h.eff.size()) * sizeof(double));
  const size_t o_fo = place(std::max<size_t>(1, h.fo.size()) * sizeof(double));
  const size_t o_srp = place(h.sr_ptr.size() * sizeof(int));
  const size_t o_sri = place(std::max<size_t>(1, h.sr_idx.size()) * sizeof(int));
  const size_t o_srn = place(std::max<size_t>(1, h.sr_nu.size()) * sizeof(double));
  const size_t o_zgp = place(h.zg_ptr.size() * sizeof(int));
  const size_t o_zgd = place(std::max<size_t>(1, h.zg_dst.size()) * sizeof(int));
  const size_t o_zgs = place(std::max<size_t>(1, h.zg_src.size()) * sizeof(int));
  const size_t o_zgs2 = place(std::max<size_t>(1, h.zg_src2.size()) * sizeof(int));
  const size_t o_zgc = place(std::max<size_t>(1, h.zg_coef.size()) * sizeof(double));
  const size_t o_prp = place(h.pr_ptr.size() * sizeof(int));
  const size_t o_prd = place(std::max<size_t>(1, h.pr_pd.size()) * sizeof(int));
  const size_t o_prn = place(std::max<size_t>(1, h.pr_nu.size()) * sizeof(double));
  const size_t o_prr = place(std::max<size_t>(1, h.pr_row.size()) * sizeof(int));
  const size_t o_prs = place(std::max<size_t>(1, h.pr_rows.size()) * sizeof(int));
  const size_t o_ord = place(h.order.size() * sizeof(int));
  const size_t o_clp = place(h.cl_ptr.size() * sizeof(int));
  const size_t o_cls = place(std::max<size_t>(1, h.cl_src.size()) * sizeof(int));
  const size_t o_clr = place(std::max<size_t>(1, h.cl_rx.size()) * sizeof(int));
  const size_t total = off;
  std::vector<char> img(total, 0);
  auto put = [&](size_t o, const void* src, size_t bytes) { if (bytes) std::memcpy(img.data() + o, src, bytes); };
  put(o_sp, h.sp.data(), h.sp.size() * sizeof(double));
  put(o_rxd, h.rxd.data(), h.rxd.size() * sizeof(double));
  put(o_rxi, h.rxi.data(), h.rxi.size() * sizeof(int));
  put(o_dnu, h.dnu.data(), h.dnu.size() * sizeof(int));
  put(o_eff, h.eff.data(), h.eff.size() * sizeof(double));
  put(o_fo, h.fo.data(), h.fo.size() * sizeof(double));
  put(o_srp, h.sr_ptr.data(), h.sr_ptr.size() * sizeof(int));
  put(o_sri, h.sr_idx.data(), h.sr_idx.size() * sizeof(int));
  put(o_srn, h.sr_nu.data(), h.sr_nu.size() * sizeof(double));
  put(o_zgp, h.zg_ptr.data(), h.zg_ptr.size() * sizeof(int));
  put(o_zgd, h.zg_dst.data(), h.zg_dst.size() * sizeof(int));
  put(o_zgs, h.zg_src.data(), h.zg_src.size() * sizeof(int));
  put(o_zgs2, h.zg_src2.data(), h.zg_src2.size() * sizeof(int));
  put(o_zgc, h.zg_coef.data(), h.zg_coef.size() * sizeof(double));
  put(o_prp, h.pr_ptr.data(), h.pr_ptr.size() * sizeof(int));
  put(o_prd, h.pr_pd.data(), h.pr_pd.size() * sizeof(int));
  put(o_prn, h.pr_nu.data(), h.pr_nu.size() * sizeof(double));
  put(o_prr, h.pr_row.data(), h.pr_row.size() * sizeof(int));
  put(o_prs, h.pr_rows.data(), h.pr_rows.size() * sizeof(int));
  put(o_ord, h.order.data(), h.order.size() * sizeof(int));
  put(o_clp, h.cl_ptr.data(), h.cl_ptr.size() * sizeof(int));
  put(o_cls, h.cl_src.data(), h.cl_src.size() * sizeof(int));
  put(o_clr, h.cl_rx.data(), h.cl_rx.size() * sizeof(int));
  e = cudaMalloc(&m->dbuf, total);
  if (e == cudaSuccess) e = cudaMemcpy(m->dbuf, img.data(), total, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_totals, 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&m->d_queue, sizeof(int));
  if (e != cudaSuccess) {
    chem_free_mechanism(m);
    return set_err(CHEM_ECUDA, std::string("chem_load_mechanism: ") + cudaGetErrorString(e));
  }
  char* b = static_cast<char*>(m->dbuf);
  DevMech& d = m->dev;
  d.K = h.K; d.R = h.R; d.N = h.K;
  d.n_elem = h.n_elem; d.n_tb = h.n_tb; d.n_fo = h.n_fo; d.n_pd = h.n_tb + h.n_fo;
  d.sp = reinterpret_cast<const double*>(b + o_sp);
  d.rxd = reinterpret_cast<const double*>(b + o_rxd);
  d.rxi = reinterpret_cast<const int*>(b + o_rxi);
  d.dnu = reinterpret_cast<const int*>(b + o_dnu);
  d.eff = reinterpret_cast<const double*>(b + o_eff);
  d.fo = reinterpret_cast<const double*>(b + o_fo);
  d.sr_ptr = reinterpret_cast<const int*>(b + o_srp);
  d.sr_idx = reinterpret_cast<const int*>(b + o_sri);
  d.sr_nu = reinterpret_cast<const double*>(b + o_srn);
  d.zg_entries = (int)h.zg_dst.size();
  d.zg_ptr = reinterpret_cast<const int*>(b + o_zgp);
  d.zg_dst = reinterpret_cast<const int*>(b + o_zgd);
  d.zg_src = reinterpret_cast<const int*>(b + o_zgs);
  d.zg_src2 = reinterpret_cast<const int*>(b + o_zgs2);
  d.zg_coef = reinterpret_cast<const double*>(b + o_zgc);
  d.pr_ptr = reinterpret_cast<const int*>(b + o_prp);
  d.pr_pd = reinterpret_cast<const int*>(b + o_prd);
  d.pr_nu = reinterpret_cast<const double*>(b + o_prn);
  d.pr_row = reinterpret_cast<const int*>(b + o_prr);
  d.pr_rows = reinterpret_cast<const int*>(b + o_prs);
  d.order = reinterpret_cast<const int*>(b + o_ord);
  d.cl_ptr = reinterpret_cast<const int*>(b + o_clp);
  d.cl_src = reinterpret_cast<const int*>(b + o_cls);
  d.cl_rx = reinterpret_cast<const int*>(b + o_clr);
  d.n_pairs = (int)h.pr_pd.size();
  d.n_prows = (int)h.pr_rows.size();
  if (d.n_pairs > 8 * (((h.K + 1) / 2) * 2)) {
    chem_free_mechanism(m);
    return set_err(CHEM_ESIZE, "chem_load_mechanism: too many pressure-dependent (row, reaction) pairs");
  }
  if ((size_t)make_plan(h.K, h.R, d.n_pd, 4).total * sizeof(double) > m->max_smem) {
    chem_free_mechanism(m);
    return set_err(CHEM_ESIZE, "chem_load_mechanism: mechanism too large for one CTA's shared memory");
  }
  *out = m;
  return CHEM_OK;
}

void chem_free_mechanism(chem_mech* m) {
  if (!m) return;
  if (m->graph.exec) cudaGraphExecDestroy(m->graph.exec);
  if (m->graph.capture_stream) cudaStreamDestroy(m->graph.capture_stream);
  cudaFree(m->dbuf);
  cudaFree(m->d_totals);
  cudaFree(m->d_queue);
  cudaFree(m->d_steps);
  cudaFree(m->d_rej);
  cudaFree(m->d_stage);
  cudaFree(m->d_adj_ws);
  cudaFree(m->d_adj_counters);
  cudaFree(m->d_map_ws);
  delete m;
}

int chem_mech_dims(const chem_mech* m, int* K, int* R) {
  if (!m) return set_err(CHEM_EINVAL, "chem_mech_dims: NULL mechanism");
  if (K) *K = m->host.K;
  if (R) *R = m->host.R;
  return CHEM_OK;
}

static int rates_or_jacobian(const chem_mech* mc, double p_Pa, const double* T, const double* Y, int64_t ncells,
                             double* f, double* J, void* stream) {
  chem_mech* m = const_cast<chem_mech*>(mc);
  if (ncells < 0) return set_err(CHEM_EINVAL, "ncells < 0");
  if (!m || (ncells > 0 && (!T || !Y || (!f && !J))))
    return set_err(CHEM_EINVAL, "chem_rates/chem_jacobian: NULL argument");
  if (!(p_Pa > 0.0)) return set_err(CHEM_EINVAL, "pressure must be positive");
  if (ncells == 0) return CHEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int N = m->host.K;
  const bool dev = is_device_ptr(T);
  const double *dT = T, *dY = Y;
  double *df = f, *dJ = J;
  if (!dev) {
    const size_t nT = ncells, nY = (size_t)N * ncells, nf = f ? (size_t)N * ncells : 0,
                 nJ = J ? (size_t)N * N * ncells : 0;
    int rc = ensure_stage(m, sizeof(double) * (nT + nY + nf + nJ));
    if (rc) return rc;
    double* s = static_cast<double*>(m->d_stage);
    double* sT = s;
    double* sY = sT + nT;
    double* sf = sY + nY;
    double* sJ = sf + nf;
    CK(cudaMemcpyAsync(sT, T, sizeof(double) * nT, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sY, Y, sizeof(double) * nY, cudaMemcpyHostToDevice, st));
    dT = sT; dY = sY;
    df = f ? sf : nullptr;
    dJ = J ? sJ : nullptr;
  }
  Launch L;
  int rc = pick_launch(m, ncells, 0, 0, 0, false, L);
  if (rc) return rc;
  switch (L.G) {
    case 1: rates_kernel<1><<<L.grid, L.threads, L.smem, st>>>(m->dev, L.plan, p_Pa * 10.0, dT, dY, ncells, df, dJ); break;
    case 2: rates_kernel<2><<<L.grid, L.threads, L.smem, st>>>(m->dev, L.plan, p_Pa * 10.0, dT, dY, ncells, df, dJ); break;
    case 4: rates_kernel<4><<<L.grid, L.threads, L.smem, st>>>(m->dev, L.plan, p_Pa * 10.0, dT, dY, ncells, df, dJ); break;
    default: rates_kernel<8><<<L.grid, L.threads, L.smem, st>>>(m->dev, L.plan, p_Pa * 10.0, dT, dY, ncells, df, dJ); break;
  }
  CK(cudaGetLastError());
  if (!dev) {
    if (f) CK(cudaMemcpyAsync(f, df, sizeof(double) * N * ncells, cudaMemcpyDeviceToHost, st));
    if (J) CK(cudaMemcpyAsync(J, dJ, sizeof(double) * N * N * ncells, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return CHEM_OK;
}

int chem_rates(const chem_mech* m, double p_Pa, const double* T, const double* Y, int64_t ncells, double* dPhidt,
               void* stream) {
  if (!dPhidt && ncells > 0) return set_err(CHEM_EINVAL, "chem_rates: NULL output");
  return rates_or_jacobian(m, p_Pa, T, Y, ncells, dPhidt, nullptr, stream);
}

int chem_jacobian(const chem_mech* m, double p_Pa, const double* T, const double* Y, int64_t ncells, double* J,
                  void* stream) {
  if (!J && ncells > 0) return set_err(CHEM_EINVAL, "chem_jacobian: NULL output");
  return rates_or_jacobian(m, p_Pa, T, Y, ncells, nullptr, J, stream);
}

static int integrate_impl(const chem_mech* mc, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                          double rtol, double atol, double* h_inout, int32_t* status, const chem_opts* opts,
                          chem_stats* stats, void* stream, double* rec, int rec_cap,
                          const double* p_cells = nullptr) {
  chem_mech* m = const_cast<chem_mech*>(mc);
  if (ncells < 0) return set_err(CHEM_EINVAL, "chem_integrate: ncells < 0");
  if (!m || (ncells > 0 && (!T || !Y))) return set_err(CHEM_EINVAL, "chem_integrate: NULL argument");
  if (ncells > (int64_t)0x7fffffff) return set_err(CHEM_EINVAL, "chem_integrate: ncells above 2^31-1");
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol >= 0.0) || !(p_Pa > 0.0))
    return set_err(CHEM_EINVAL, "chem_integrate: dt, rtol and p must be positive, atol non-negative");
  chem_opts o;
  chem_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_steps < 1) return set_err(CHEM_EINVAL, "chem_integrate: max_steps < 1");
  if (o.precision != CHEM_PREC_FP64 && o.precision != CHEM_PREC_MIXED &&
      o.precision != CHEM_PREC_MIXED_FF)
    return set_err(CHEM_EINVAL, "chem_integrate: unknown precision mode");
  if (o.precision == CHEM_PREC_MIXED && (o.refine_sweeps < 1 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate: refine_sweeps must be 1..4");
  if (o.precision == CHEM_PREC_MIXED_FF && (o.refine_sweeps < 0 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate: refine_sweeps must be 0..4");
  if (o.solver != CHEM_SOLVER_ROSENBROCK && o.solver != CHEM_SOLVER_SEULEX)
    return set_err(CHEM_EINVAL, "chem_integrate: unknown solver");
  if (o.solver == CHEM_SOLVER_SEULEX && (o.precision != CHEM_PREC_FP64 || rec))
    return set_err(CHEM_EINVAL, "chem_integrate: Seulex runs in FP64 and without step records");
  if (o.jacobian != CHEM_JAC_ANALYTIC && o.jacobian != CHEM_JAC_FD)
    return set_err(CHEM_EINVAL, "chem_integrate: unknown Jacobian mode");
  if (o.jacobian == CHEM_JAC_FD && (o.solver != CHEM_SOLVER_ROSENBROCK || rec))
    return set_err(CHEM_EINVAL, "chem_integrate: the finite-difference Jacobian serves the Rosenbrock solve only, "
                                "without step records");
  if (m->host.K > 128) return set_err(CHEM_ESIZE, "chem_integrate: more than 128 species");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (ncells == 0) return CHEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int K = m->host.K;
  int rc = ensure_cells(m, ncells);
  if (rc) return rc;
  const bool dev = is_device_ptr(T);
  double *dT = T, *dY = Y, *dh = h_inout;
  int32_t* dstat = status;
  if (!dev) {
    const size_t nT = ncells, nY = (size_t)K * ncells, nh = h_inout ? ncells : 0, ns = status ? ncells : 0;
    rc = ensure_stage(m, sizeof(double) * (nT + nY + nh) + sizeof(int32_t) * ns + 16);
    if (rc) return rc;
    double* s = static_cast<double*>(m->d_stage);
    dT = s;
    dY = s + nT;
    dh = h_inout ? dY + nY : nullptr;
    dstat = status ? reinterpret_cast<int32_t*>(dY + nY + nh) : nullptr;
    CK(cudaMemcpyAsync(dT, T, sizeof(double) * nT, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dY, Y, sizeof(double) * nY, cudaMemcpyHostToDevice, st));
    if (h_inout) CK(cudaMemcpyAsync(dh, h_inout, sizeof(double) * nh, cudaMemcpyHostToDevice, st));
  }
  IntegrateArgs a;
  std::memset(&a, 0, sizeof(a));  // padding too: the graph cache compares whole argument sets
  a.p = p_Pa * 10.0; a.dt = dt; a.rtol = rtol; a.atol = atol;
  a.T = dT; a.Y = dY; a.h_inout = dh; a.status = dstat;
  a.steps_out = m->d_steps; a.rej_out = m->d_rej;
  a.totals = m->d_totals; a.queue = m->d_queue;
  a.ncells = ncells; a.first = 0; a.count = ncells; a.max_steps = o.max_steps; a.use_queue = o.use_queue;
  a.mixed = o.precision == CHEM_PREC_MIXED ? 1 : o.precision == CHEM_PREC_MIXED_FF ? 2 : 0;
  a.refine_sweeps = o.refine_sweeps;
  a.rec = rec; a.rec_cap = rec_cap;
  a.solver = o.solver;
  a.fdjac = o.jacobian == CHEM_JAC_FD;
  a.p_cells = p_cells;
  if (o.use_graph && dev) {
    rc = launch_via_graph(m, o, a, st);
  } else {
    rc = enqueue_integrate(m, o, a, st);
  }
  if (rc) return rc;
  if (!dev) {
    CK(cudaMemcpyAsync(T, dT, sizeof(double) * ncells, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Y, dY, sizeof(double) * K * ncells, cudaMemcpyDeviceToHost, st));
    if (h_inout) CK(cudaMemcpyAsync(h_inout, dh, sizeof(double) * ncells, cudaMemcpyDeviceToHost, st));
    if (status) CK(cudaMemcpyAsync(status, dstat, sizeof(int32_t) * ncells, cudaMemcpyDeviceToHost, st));
  }
  if (stats) {
    unsigned long long tot[4];
    CK(cudaMemcpyAsync(tot, m->d_totals, sizeof(tot), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stats->steps = (int64_t)tot[0];
    stats->rejects = (int64_t)tot[1];
    stats->failed_cells = (int64_t)tot[2];
    stats->refine_fallbacks = (int64_t)tot[3];
  } else if (!dev) {
    CK(cudaStreamSynchronize(st));
  }
  return CHEM_OK;
}

int chem_integrate(const chem_mech* m, double p_Pa, double* T, double* Y, int64_t ncells, double dt, double rtol,
                   double atol, double* h_inout, int32_t* status, const chem_opts* opts, chem_stats* stats,
                   void* stream) {
  return integrate_impl(m, p_Pa, T, Y, ncells, dt, rtol, atol, h_inout, status, opts, stats, stream, nullptr, 0);
}

int chem_integrate_varp(const chem_mech* m, const double* p_Pa, double* T, double* Y, int64_t ncells, double dt,
                        double rtol, double atol, double* h_inout, int32_t* status, const chem_opts* opts,
                        chem_stats* stats, void* stream) {
  if (!m) return set_err(CHEM_EINVAL, "chem_integrate_varp: NULL mechanism");
  if (ncells < 0) return set_err(CHEM_EINVAL, "chem_integrate_varp: ncells < 0");
  if (ncells == 0) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return CHEM_OK;
  }
  if (!p_Pa || !T || !Y) return set_err(CHEM_EINVAL, "chem_integrate_varp: NULL argument");
  const void* arrays[5] = {p_Pa, T, Y, h_inout, status};
  for (const void* ptr : arrays)
    if (ptr && !is_device_ptr(ptr)) return set_err(CHEM_EINVAL, "chem_integrate_varp: device arrays only");
  // the scalar pressure only passes the argument check; every cell uses its own p_Pa[c]
  return integrate_impl(m, 1.0, T, Y, ncells, dt, rtol, atol, h_inout, status, opts, stats, stream, nullptr, 0, p_Pa);
}

int chem_integrate_mapped(const chem_mech* mc, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                          double rtol, double atol, double* h_inout, int32_t* status, const double* refs,
                          int32_t n_ref, double tol_T, double tol_Y, int32_t* zone, int64_t* n_mapped,
                          const chem_opts* opts, chem_stats* stats, void* stream) {
  chem_mech* m = const_cast<chem_mech*>(mc);
  if (!m) return set_err(CHEM_EINVAL, "chem_integrate_mapped: NULL mechanism");
  if (ncells < 0 || ncells > (int64_t)0x7fffffff) return set_err(CHEM_EINVAL, "chem_integrate_mapped: bad ncells");
  if (n_ref < 0 || n_ref > 64 || (n_ref > 0 && !refs))
    return set_err(CHEM_EINVAL, "chem_integrate_mapped: 0..64 reference states, host array");
  if (!(tol_T >= 0.0) || !(tol_Y >= 0.0)) return set_err(CHEM_EINVAL, "chem_integrate_mapped: negative tolerance");
  if (n_mapped) *n_mapped = 0;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (ncells == 0) return CHEM_OK;
  if (!T || !Y) return set_err(CHEM_EINVAL, "chem_integrate_mapped: NULL argument");
  const void* arrays[5] = {T, Y, h_inout, status, zone};
  for (const void* ptr : arrays)
    if (ptr && !is_device_ptr(ptr)) return set_err(CHEM_EINVAL, "chem_integrate_mapped: device arrays only");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int K = m->host.K;
  const int64_t nc_max = ncells + n_ref;
  // workspace: refs | count | zone | pos | list | Tc | Yc | hc | sc
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
  const size_t o_refs = place(sizeof(double) * (size_t)std::max(n_ref, 1) * (1 + K));
  const size_t o_cnt = place(sizeof(unsigned long long));
  const size_t o_zone = place(sizeof(int32_t) * ncells);
  const size_t o_pos = place(sizeof(int64_t) * ncells);
  const size_t o_list = place(sizeof(int64_t) * ncells);
  const size_t o_Tc = place(sizeof(double) * nc_max);
  const size_t o_Yc = place(sizeof(double) * nc_max * K);
  const size_t o_hc = place(sizeof(double) * nc_max);
  const size_t o_sc = place(sizeof(int32_t) * nc_max);
  if (off > m->cap_map_ws) {
    cudaFree(m->d_map_ws);
    m->d_map_ws = nullptr;
    m->cap_map_ws = 0;
    CK(cudaMalloc(&m->d_map_ws, off));
    m->cap_map_ws = off;
  }
  char* b = static_cast<char*>(m->d_map_ws);
  double* d_refs = reinterpret_cast<double*>(b + o_refs);
  unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(b + o_cnt);
  int32_t* d_zone = zone ? zone : reinterpret_cast<int32_t*>(b + o_zone);
  int64_t* d_pos = reinterpret_cast<int64_t*>(b + o_pos);
  int64_t* d_list = reinterpret_cast<int64_t*>(b + o_list);
  double* Tc = reinterpret_cast<double*>(b + o_Tc);
  double* Yc = reinterpret_cast<double*>(b + o_Yc);
  double* hc = reinterpret_cast<double*>(b + o_hc);
  int32_t* sc = reinterpret_cast<int32_t*>(b + o_sc);
  if (n_ref > 0)
    CK(cudaMemcpyAsync(d_refs, refs, sizeof(double) * (size_t)n_ref * (1 + K), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st));
  const int threads = 256;
  const unsigned blocks = (unsigned)((ncells + threads - 1) / threads);
  map_classify_kernel<<<blocks, threads, 0, st>>>(T, Y, ncells, K, d_refs, n_ref, tol_T, tol_Y, d_zone, d_pos,
                                                  d_list, d_cnt);
  CK(cudaGetLastError());
  unsigned long long n_un_u = 0;
  CK(cudaMemcpyAsync(&n_un_u, d_cnt, sizeof(n_un_u), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));  // the solve's size is the number of cells left to solve
  const int64_t n_un = (int64_t)n_un_u;
  const int64_t nc = n_un + n_ref;
  if (nc > 0) {
    map_gather_kernel<<<(unsigned)((nc + threads - 1) / threads), threads, 0, st>>>(T, Y, h_inout, ncells, K, d_refs,
                                                                                   n_ref, d_list, n_un, Tc, Yc, hc);
    CK(cudaGetLastError());
    chem_opts o;
    chem_default_opts(&o);
    if (opts) o = *opts;
    o.use_graph = 0;  // the compact arrays' size changes from call to call
    const int rc = integrate_impl(m, p_Pa, Tc, Yc, nc, dt, rtol, atol, hc, sc, &o, stats, stream, nullptr, 0);
    if (rc) return rc;
  }
  map_scatter_kernel<<<blocks, threads, 0, st>>>(T, Y, h_inout, status, ncells, K, d_refs, d_zone, d_pos, n_un, n_ref,
                                                 Tc, Yc, hc, sc);
  CK(cudaGetLastError());
  if (n_mapped) *n_mapped = ncells - n_un;
  return CHEM_OK;
}

int chem_integrate_record(const chem_mech* m, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                          double rtol, double atol, double* h_inout, int32_t* status, double* rec,
                          int32_t max_steps_rec, int32_t* nsteps, const chem_opts* opts, chem_stats* stats,
                          void* stream) {
  if (!m) return set_err(CHEM_EINVAL, "chem_integrate_record: NULL mechanism");
  if (ncells < 0) return set_err(CHEM_EINVAL, "chem_integrate_record: ncells < 0");
  if (max_steps_rec < 1) return set_err(CHEM_EINVAL, "chem_integrate_record: max_steps_rec < 1");
  if (opts && opts->precision != CHEM_PREC_FP64)
    return set_err(CHEM_EINVAL, "chem_integrate_record: record mode integrates in FP64 only");
  if (ncells == 0) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return CHEM_OK;
  }
  if (!rec || !status || !nsteps || !T || !Y) return set_err(CHEM_EINVAL, "chem_integrate_record: NULL argument");
  const void* arrays[6] = {T, Y, h_inout, status, rec, nsteps};
  for (const void* ptr : arrays)
    if (ptr && !is_device_ptr(ptr)) return set_err(CHEM_EINVAL, "chem_integrate_record: device arrays only");
  int rc = integrate_impl(m, p_Pa, T, Y, ncells, dt, rtol, atol, h_inout, status, opts, stats, stream, rec,
                          max_steps_rec);
  if (rc) return rc;
  CK(cudaMemcpyAsync(nsteps, m->d_steps, sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice,
                     static_cast<cudaStream_t>(stream)));
  return CHEM_OK;
}

int chem_adjoint(const chem_mech* mc, double p_Pa, int64_t ncells, const double* rec, int32_t max_steps_rec,
                 const int32_t* nsteps, const int32_t* status, const double* gT, const double* gY, double* gT0,
                 double* gY0, double* g_lnA, double* g_lnA_cells, void* stream) {
  chem_mech* m = const_cast<chem_mech*>(mc);
  if (!m) return set_err(CHEM_EINVAL, "chem_adjoint: NULL mechanism");
  if (ncells < 0 || ncells > (int64_t)0x7fffffff) return set_err(CHEM_EINVAL, "chem_adjoint: bad ncells");
  if (max_steps_rec < 1) return set_err(CHEM_EINVAL, "chem_adjoint: max_steps_rec < 1");
  if (!(p_Pa > 0.0)) return set_err(CHEM_EINVAL, "chem_adjoint: pressure must be positive");
  if (m->host.K > 128) return set_err(CHEM_ESIZE, "chem_adjoint: more than 128 species");
  if (ncells == 0) return CHEM_OK;
  if (!rec || !nsteps || !status || !gT || !gY || !gT0 || !gY0)
    return set_err(CHEM_EINVAL, "chem_adjoint: NULL argument");
  const void* arrays[9] = {rec, nsteps, status, gT, gY, gT0, gY0, g_lnA, g_lnA_cells};
  for (const void* ptr : arrays)
    if (ptr && !is_device_ptr(ptr)) return set_err(CHEM_EINVAL, "chem_adjoint: device arrays only");
  const size_t need = adjoint_workspace_doubles(m->host.R, ncells, g_lnA_cells != nullptr);
  if (need > m->cap_adj_ws) {
    cudaFree(m->d_adj_ws);
    m->d_adj_ws = nullptr;
    m->cap_adj_ws = 0;
    CK(cudaMalloc(&m->d_adj_ws, need * sizeof(double)));
    m->cap_adj_ws = need;
  }
  if (!m->d_adj_counters) CK(cudaMalloc(&m->d_adj_counters, 2 * sizeof(int)));
  std::string err;
  const int rc = adjoint_enqueue(m->dev, m->num_sms, m->max_smem, p_Pa * 10.0, ncells, rec, max_steps_rec, nsteps,
                                 status, gT, gY, gT0, gY0, g_lnA, g_lnA_cells, m->d_adj_ws, m->d_adj_counters,
                                 static_cast<cudaStream_t>(stream), err);
  if (rc) return set_err(rc, err);
  return CHEM_OK;
}

int chem_get_lnA(const chem_mech* m, double* lnA) {
  if (!m || !lnA) return set_err(CHEM_EINVAL, "chem_get_lnA: NULL argument");
  const HostMech& h = m->host;
  for (int dr = 0; dr < h.R; ++dr) lnA[h.order[dr]] = h.rxd[(size_t)dr * kRxDoubles];
  return CHEM_OK;
}

int chem_set_lnA(chem_mech* m, const double* lnA) {
  if (!m || !lnA) return set_err(CHEM_EINVAL, "chem_set_lnA: NULL argument");
  HostMech& h = m->host;
  for (int r = 0; r < h.R; ++r)
    if (!std::isfinite(lnA[r])) return set_err(CHEM_EINVAL, "chem_set_lnA: non-finite value");
  for (int dr = 0; dr < h.R; ++dr) h.rxd[(size_t)dr * kRxDoubles] = lnA[h.order[dr]];
  // the device tables are read by kernels in flight on any stream: wait for them first
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(const_cast<double*>(m->dev.rxd), h.rxd.data(), h.rxd.size() * sizeof(double),
                cudaMemcpyHostToDevice));
  return CHEM_OK;
}

#ifdef CHEM_PHASE_TIMERS
// Debug builds only: per-phase cycle totals {rates+J data, J assembly, W+LU, solves, stage
// rates, control} summed over cell groups since the last call; resets them.
int chem_debug_phase_cycles(unsigned long long* out8) {
  CK(cudaMemcpyFromSymbol(out8, g_phase_cycles, sizeof(unsigned long long) * 8));
  unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  CK(cudaMemcpyToSymbol(g_phase_cycles, z, sizeof(z)));
  return CHEM_OK;
}
#endif

// Device address of g_noalloc_scratch on the current device, looked up once per device (the
// host-side name of a __device__ array is only a stand-in, never a device address).
static int noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* addr[256] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return set_err(CHEM_ECUDA, "chem_integrate_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_err(CHEM_ECUDA, std::string("chem_integrate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    addr[dev] = p;
  }
  *out = addr[dev];
  return CHEM_OK;
}

int chem_integrate_noalloc(const chem_mech* mc, double p_Pa, double* T, double* Y, int64_t ncells, double dt,
                           double rtol, double atol, double* h_inout, int32_t* status, int32_t* steps,
                           int32_t* rejects, const chem_opts* opts, chem_stats* stats, void* stream) {
  chem_mech* m = const_cast<chem_mech*>(mc);
  if (ncells < 0) return set_err(CHEM_EINVAL, "chem_integrate_noalloc: ncells < 0");
  if (ncells > kNoAllocMaxCells)
    return set_err(CHEM_ESIZE, "chem_integrate_noalloc: " + std::to_string(ncells) + " cells exceed its fixed scratch of " +
                                   std::to_string(kNoAllocMaxCells) + " cells; use chem_integrate");
  if (!m || (ncells > 0 && (!T || !Y))) return set_err(CHEM_EINVAL, "chem_integrate_noalloc: NULL argument");
  if (!(dt > 0.0) || !(rtol > 0.0) || !(atol >= 0.0) || !(p_Pa > 0.0))
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: dt, rtol and p must be positive, atol non-negative");
  chem_opts o;
  chem_default_opts(&o);
  if (opts) o = *opts;
  if (o.max_steps < 1) return set_err(CHEM_EINVAL, "chem_integrate_noalloc: max_steps < 1");
  if (o.precision != CHEM_PREC_FP64 && o.precision != CHEM_PREC_MIXED &&
      o.precision != CHEM_PREC_MIXED_FF)
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: unknown precision mode");
  if (o.precision == CHEM_PREC_MIXED && (o.refine_sweeps < 1 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: refine_sweeps must be 1..4");
  if (o.precision == CHEM_PREC_MIXED_FF && (o.refine_sweeps < 0 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: refine_sweeps must be 0..4");
  if (o.solver != CHEM_SOLVER_ROSENBROCK && o.solver != CHEM_SOLVER_SEULEX)
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: unknown solver");
  if (o.solver == CHEM_SOLVER_SEULEX && o.precision != CHEM_PREC_FP64)
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: Seulex runs in FP64");
  if (o.jacobian != CHEM_JAC_ANALYTIC && (o.jacobian != CHEM_JAC_FD || o.solver != CHEM_SOLVER_ROSENBROCK))
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: bad Jacobian mode");
  if (m->host.K > 128) return set_err(CHEM_ESIZE, "chem_integrate_noalloc: more than 128 species");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (ncells == 0) return CHEM_OK;
  const void* arrays[6] = {T, Y, h_inout, status, steps, rejects};
  for (const void* ptr : arrays)
    if (ptr && !is_device_ptr(ptr))
      return set_err(CHEM_EINVAL, "chem_integrate_noalloc: every array must be device memory (host arrays would "
                                  "need a staging allocation)");
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* s = static_cast<unsigned char*>(scratch);
  CK(cudaMemsetAsync(s, 0, kNoAllocCounters, st));  // queue counter and totals start at zero
  Launch L;
  rc = pick_launch(m, ncells, o.warps_per_cell, o.cells_per_cta, o.ctas_per_sm, true, L, o.solver);
  if (rc) return rc;
  int32_t* d_steps = reinterpret_cast<int32_t*>(s + kNoAllocCounters);
  int32_t* d_rej = d_steps + kNoAllocMaxCells;
  IntegrateArgs a;
  std::memset(&a, 0, sizeof(a));
  a.p = p_Pa * 10.0; a.dt = dt; a.rtol = rtol; a.atol = atol;
  a.T = T; a.Y = Y; a.h_inout = h_inout; a.status = status;
  a.steps_out = d_steps; a.rej_out = d_rej;
  a.totals = reinterpret_cast<unsigned long long*>(s + 64);
  a.queue = reinterpret_cast<int*>(s);
  a.ncells = ncells; a.first = 0; a.count = ncells; a.max_steps = o.max_steps; a.use_queue = o.use_queue;
  a.mixed = o.precision == CHEM_PREC_MIXED ? 1 : o.precision == CHEM_PREC_MIXED_FF ? 2 : 0;
  a.refine_sweeps = o.refine_sweeps;
  a.solver = o.solver;
  a.fdjac = o.jacobian == CHEM_JAC_FD;
  launch_integrate(L, st, m->dev, a);
  CK(cudaGetLastError());
  if (steps) CK(cudaMemcpyAsync(steps, d_steps, sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice, st));
  if (rejects) CK(cudaMemcpyAsync(rejects, d_rej, sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice, st));
  if (stats) {
    unsigned long long tot[4];
    CK(cudaMemcpyAsync(tot, a.totals, sizeof(tot), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    stats->steps = (int64_t)tot[0];
    stats->rejects = (int64_t)tot[1];
    stats->failed_cells = (int64_t)tot[2];
    stats->refine_fallbacks = (int64_t)tot[3];
  }
  return CHEM_OK;
}

int chem_debug_exp(const double* x, double* y, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return set_err(CHEM_EINVAL, "chem_debug_exp: bad arguments");
  if (n == 0) return CHEM_OK;
  if (!is_device_ptr(x) || !is_device_ptr(y)) return set_err(CHEM_EINVAL, "chem_debug_exp: device arrays only");
  const int threads = 256;
  const int64_t blocks = (n + threads - 1) / threads;
  exp_probe_kernel<<<(unsigned)blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(x, y, n);
  CK(cudaGetLastError());
  return CHEM_OK;
}

int chem_probe_fp64_peak(double* tflops) {
  if (!tflops) return set_err(CHEM_EINVAL, "chem_probe_fp64_peak: NULL output");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 4, threads = 256, iters = 8192;
  double* buf = nullptr;
  CK(cudaMalloc(&buf, sizeof(double) * blocks * threads));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fp64_peak_kernel<<<blocks, threads>>>(buf, iters / 8, 0.999);  // warm-up
  cudaEventRecord(e0);
  fp64_peak_kernel<<<blocks, threads>>>(buf, iters, 0.999);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return set_err(CHEM_ECUDA, std::string("chem_probe_fp64_peak: ") + cudaGetErrorString(e));
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return CHEM_OK;
}

int chem_last_cell_counters(const chem_mech* m, int32_t* steps, int32_t* rejects, int64_t ncells, void* stream) {
  if (!m) return set_err(CHEM_EINVAL, "chem_last_cell_counters: NULL mechanism");
  if (ncells < 0 || ncells > m->cap_cells) return set_err(CHEM_EINVAL, "chem_last_cell_counters: bad ncells");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (steps) CK(cudaMemcpyAsync(steps, m->d_steps, sizeof(int32_t) * ncells, cudaMemcpyDefault, st));
  if (rejects) CK(cudaMemcpyAsync(rejects, m->d_rej, sizeof(int32_t) * ncells, cudaMemcpyDefault, st));
  CK(cudaStreamSynchronize(st));
  return CHEM_OK;
}

}  // extern "C"
