// Device code of the integrate kernels: the Rosenbrock solve (integrate_kernel) and Seulex
// (seulex_kernel), with the forward-difference Jacobian and the low-precision factorisations.
// Included by one translation unit per cell-group width G (integrate_g*.cu), each of which
// instantiates the kernels for its G and defines the launchers of integrate.h.
#pragma once
#include <cuda_runtime.h>

#include "../../include/chemgpu.h"
#include "cell_device.cuh"
#include "chem_internal.h"
#include "integrate.h"

namespace {
// ------------------------------------------------------------------------------------------
// Optional per-phase cycle counters (compile with -DCHEM_PHASE_TIMERS): thread 0 of each cell
// group accumulates clock64() deltas per phase into IntegrateArgs::phase; read with
// chem_debug_phase_cycles().

#ifdef CHEM_PHASE_TIMERS
#define PHASE_BEGIN long long ph_t0_ = clock64();
#define PHASE_END(slot)                                                  \
  do {                                                                    \
    long long ph_t1_ = clock64();                                         \
    if (g.t == 0 && a.phase) atomicAdd(&a.phase[slot], (unsigned long long)(ph_t1_ - ph_t0_)); \
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

// Refinement stops when the last correction is below this fraction of the error-control scale
// atol + rtol |y| of every component (or the residual is at the FP64 rounding level)
#ifndef CHEM_REFINE_TOL
#define CHEM_REFINE_TOL 1e-5
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
__device__ inline float to_low<float>(double v) { return f32_of(v); }
template <>
__device__ inline FF to_low<FF>(double v) { return FF(v); }

// Equilibrate W = I gh - J by powers of two (row exponents er, then column exponents ec, from
// the largest entries) and factor S = D_r W D_c in the low precision L (FP32 or FP32 pairs) in
// buffer B; the reciprocal pivots go to invd.  The diagonal gh + (-J)_ii is formed once in FP64
// (in the residual vector, free until the stage solves), so the scans only compare exponents.
template <int G, typename L>
__device__ __forceinline__ bool form_and_factor_low(const Grp<G>& g, const CellMem& w, int N, double gh, L* invd) {
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
  return cell_lu_default<G, L>(g, S, N, w.piv, w.perm, invd);
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
__device__ __forceinline__ bool stage_solve_low(const Grp<G>& g, const CellMem& w, const IntegrateArgs& a, int N, double gh,
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
      c = Grp<G>::nanmax(c, fabs(d) * w.err[i]);  // w.err: 1 / (atol + rtol |y|), set per attempt
    }
    conv = g.max_nan_any(c, above);
    if (!above && conv == conv) conv = 0.0;  // residual at the FP64 rounding level
    if (conv <= CHEM_REFINE_TOL) break;
  }
  return conv <= CHEM_REFINE_TOL;
}

// u <- W^-1 rhs: FP64 factors (lowp 0: one solve), FP32 factors (1) or FP32 pairs (2).
template <int G>
__device__ __forceinline__ bool stage_solve(const Grp<G>& g, const CellMem& w, const IntegrateArgs& a, int N, double gh, int lowp,
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
        if (lowp) {
          // reciprocal error-control scales of the refinement's stopping test (the error vector is
          // free until the stages are combined)
          for (int i = g.t; i < N; i += NT) w.err[i] = 1.0 / (a.atol + a.rtol * fabs(w.y[i]));
        }
        if (lowp == 1) {
          ok = form_and_factor_low<G, float>(g, w, N, gh, w.invd32);
        } else if (lowp == 2) {
          ok = form_and_factor_low<G, FF>(g, w, N, gh, reinterpret_cast<FF*>(w.invdiag));
        } else {
          for (int e = g.t; e < N * N; e += NT) w.B[e] = w.A[e];
          g.sync();
          for (int i = g.t; i < N; i += NT) w.B[i * N + i] += gh;
          g.sync();
          ok = cell_lu_default<G, double>(g, w.B, N, w.piv, w.perm, w.invdiag);
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
      // err^(-1/4) of the step-size factor, by one thread for the group (see cell_rates)
      double p25;
      if (G > 1) {
        if (g.t == 0) w.bc[5] = pow(err, -0.25);
        g.sync();
        p25 = w.bc[5];
      } else {
        p25 = pow(err, -0.25);
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
        fac = fmin(6.0, fmax(0.2, 0.9 * p25));
        if (last_rej) fac = fmin(fac, 1.0);
        last_rej = false;
        h_next = h * fac;
        if (t >= a.dt) break;
      } else {
        ++nrej;
        fac = (err == err && err < INFINITY) ? fmax(0.2, 0.9 * p25) : 0.2;
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
        if (!cell_lu_default<G, double>(g, w.B, N, w.piv, w.perm, w.invdiag)) { badstep = true; break; }
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

}  // namespace

// The launchers of integrate.h for one G (used once per integrate_g*.cu).
#define CHEM_DEFINE_INTEGRATE_LAUNCHERS(G)                                                          \
  namespace chemgpu {                                                                              \
  const void* integrate_kernel_fn_g##G(int solver) {                                               \
    return solver == CHEM_SOLVER_SEULEX ? (const void*)seulex_kernel<G> : (const void*)integrate_kernel<G>; \
  }                                                                                                \
  void integrate_launch_g##G(int solver, int grid, int threads, size_t smem, cudaStream_t st,      \
                             const DevMech& d, const IntegrateArgs& a) {                           \
    const Plan plan = make_plan(d.K, d.R, d.n_pd, G);                                              \
    if (solver == CHEM_SOLVER_SEULEX)                                                              \
      seulex_kernel<G><<<grid, threads, smem, st>>>(d, plan, a);                                   \
    else                                                                                           \
      integrate_kernel<G><<<grid, threads, smem, st>>>(d, plan, a);                                \
  }                                                                                                \
  }
