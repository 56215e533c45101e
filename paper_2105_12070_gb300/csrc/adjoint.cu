// Discrete adjoint of the Rosenbrock integration (reverse sweep over recorded accepted steps).
//
// The forward map of one accepted step (transformed form, W = I/(gamma h) - J(y)):
//   W u_i = f(Y_i) + sum_{j<i} (c_ij/h) u_j,   Y_i = y + sum_{j<i} a_ij u_j,
//   y_new = y + sum_i m_i u_i,
// with h frozen (the step sizes the controller chose in the forward run).  Its adjoint, given
// lambda = dL/dy_new: with ub_i = m_i lambda, for i = 4 .. 1
//   v_i = W^-T ub_i,   ub_j += (c_ij/h) v_i + a_ij J(Y_i)^T v_i   (j < i),
// and dL/dy = lambda + sum_i J(Y_i)^T v_i + sum_i (D_{u_i} J(y))^T v_i, where the last term
// differentiates W = I/(gamma h) - J(y) (D_u J = the derivative of J along u; the symmetry of
// the second derivatives of f turns grad_y (v^T J(y) u) into (D_u J)^T v).  For the parameters
// theta_r = ln A_r: dL/dtheta += sum_i v_i . df/dtheta(Y_i) + sum_i D_{u_i} (v_i . df/dtheta)(y).
// Stage 4 evaluates f at Y_3 (a_4j = a_3j), so J(Y_3) is applied once to v_3 + v_4, and
// Y_1 = y.  D_u J and D_u (v . df/dtheta) come from one evaluation of the rate and Jacobian code
// in dual numbers along u; its value part is J(y), which gives the stage-1 term J(y)^T v_1.
//
// Per accepted step and cell: one FP64 Jacobian at y_n and the LU of W (as in the solve), the
// four stages (two rate evaluations, four solves), four transposed solves, products J^T v at
// Y_3 and Y_2, and four evaluations of J^T v_i in dual numbers along u_i.  The J^T products are
// matrix-free (cell_jacobian_vjp): weighted column sums of d omega/dC built from the
// per-reaction data, so only the Jacobian at y_n (for W) is ever formed.  That keeps the working
// set near 95 KB for 53 species: two cells of 4 warps per CTA, cells from a queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/chemgpu.h"
#include "adjoint.h"
#include "cell_device.cuh"

namespace {

// Per-cell shared-memory plan of the adjoint (in doubles).
struct AdjPlan {
  int N, n2, SA, nR2, nM2, nP2, nAB2, G;
  int off_M, off_vec, off_ev, off_ab, off_tz, off_yd, off_P, off_gA, off_piv, off_red, total;
};

AdjPlan make_adj_plan(int K, int R, int n_pd, int n_pairs, int G) {
  AdjPlan p;
  p.G = G;
  p.N = K;
  p.n2 = round2(K);
  p.SA = round2(std::max(K * K, 8 * R));
  p.nR2 = round2(R);
  p.nM2 = round2(std::max(n_pd, 1));
  p.nP2 = round2(std::max(n_pairs, 1));
  p.nAB2 = round2(2 * R + 2 * n_pd);
  // matrix region, reused by the phases of a step: the Jacobian at y_n (scratch, then -J, then
  // W and its LU in place) with its Z scratch behind it; the LU with the per-reaction scratch of
  // the stage-state evaluations behind it; the dual-number per-reaction scratch
  p.off_M = 0;
  const int msize = round2(std::max({p.SA + K * K, K * K + 8 * R, 16 * R}));
  // 18 vectors: y f ys rhs u0..u3 ub0..ub3 (v_i overwrite ub_i) ybar lam invdiag wv (+2 spare)
  p.off_vec = msize;
  // evaluation arrays, sized as duals: 12 species arrays, q, [M], pair coefficients
  p.off_ev = p.off_vec + 18 * p.n2;
  p.off_ab = p.off_ev + 2 * (12 * p.n2 + p.nR2 + p.nM2 + p.nP2);
  p.off_tz = p.off_ab + 2 * p.nAB2;     // per-reaction weights of the J^T product (duals)
  p.off_yd = p.off_tz + 2 * 2 * p.n2;   // weighted column sums (duals)
  p.off_P = p.off_yd + 6 * p.n2;        // dual state, dual source term, dual J^T v
  p.off_gA = p.off_P + 2 * p.nR2;       // P_r (dual), then the cell's ln A gradient
  p.off_piv = p.off_gA + p.nR2;
  p.off_red = p.off_piv + round2(K + 2);
  p.total = round2(p.off_red + 6 * G + 2);
  return p;
}

struct AdjMem {
  double* M;
  double *y, *f, *ys, *rhs, *u[4], *v[4], *ybar, *lam, *invdiag, *wv;
  Dual *yd, *fd, *od;
  double* gA;
  int *piv, *perm, *slot;
  double* red;
  int n2;  // vector stride: u[k] = u[0] + k n2, v[k] = v[0] + k n2 (loops index them arithmetically,
           // so the pointer arrays stay in registers)
};

__device__ inline AdjMem carve_adj(double* base, const AdjPlan& p) {
  AdjMem w;
  w.M = base + p.off_M;
  double* v = base + p.off_vec;
  const int n = p.n2;
  w.y = v; w.f = v + n; w.ys = v + 2 * n; w.rhs = v + 3 * n;
  for (int i = 0; i < 4; ++i) {
    w.u[i] = v + (4 + i) * n;
    w.v[i] = v + (8 + i) * n;  // holds ub_i until the transposed solve turns it into v_i
  }
  w.ybar = v + 12 * n; w.lam = v + 13 * n; w.invdiag = v + 14 * n; w.wv = v + 15 * n;
  w.yd = reinterpret_cast<Dual*>(base + p.off_yd);
  w.fd = w.yd + n;
  w.od = w.fd + n;
  w.gA = base + p.off_gA;
  w.piv = reinterpret_cast<int*>(base + p.off_piv);
  w.perm = w.piv + p.N + 2;
  w.red = base + p.off_red;
  w.slot = reinterpret_cast<int*>(base + p.off_red + 6 * p.G);
  w.n2 = n;
  return w;
}

// The evaluation arrays as S (double for the FP64 passes, Dual for the dual-number passes; the
// double view uses the first half of the same memory).
template <class S>
__device__ inline EvalMem<S> adj_eval_mem(double* base, const AdjPlan& p) {
  S* e = reinterpret_cast<S*>(base + p.off_ev);
  const int n = p.n2;
  EvalMem<S> m;
  m.C = e; m.hRT = e + n; m.cpR = e + 2 * n; m.gRT = e + 3 * n; m.omega = e + 4 * n; m.dcpR = e + 5 * n;
  m.zc = e + 6 * n; m.dwT = e + 7 * n; m.rowA = e + 8 * n; m.rowB = e + 9 * n; m.ccol = e + 10 * n; m.wq = e + 11 * n;
  m.q = e + 12 * n;
  m.M = m.q + p.nR2;
  m.pv = m.M + p.nM2;
  return m;
}

template <int G>
__device__ inline void solve_t(const Grp<G>& g, const AdjMem& w, int N, double* x) {
  if (g.warp() == g.lead) warp_lu_solve_t(w.M, N, w.perm, w.invdiag, x, x);
  g.sync();
}

// One accepted step backwards: w.y = y_n, h = h_n, w.lam = dL/dy_{n+1} on entry; dL/dy_n in
// w.lam and the step's ln A terms added to w.gA on exit.  False if W is exactly singular.
template <int G>
__device__ bool adjoint_step(const DevMech& m, const Grp<G>& g, const AdjPlan& plan, double p, double h,
                             const AdjMem& w, const EvalMem<double>& ed, const EvalMem<Dual>& eD, double* abd,
                             Dual* abD, double* tzd, Dual* tzD, double* Pd, Dual* PD) {
  constexpr int NT = Grp<G>::NT;
  const int N = m.N, R = m.R;
  const double gh = 1.0 / (c_gamma * h);
  const double invh = 1.0 / h;
  double* LU = w.M;            // -J(y_n), then W, then its factors
  double* scr = w.M + N * N;   // per-reaction scratch of the stage-state evaluations
  // J(y) and the factors of W (as in the solve)
  const CellScalars s0 = cell_rates(m, g, p, w.y, w.f, ed, LU, true);
  cell_jacobian(m, g, s0, w.f, ed, LU, w.M + plan.SA);
  for (int i = g.t; i < N; i += NT) LU[i * N + i] += gh;
  g.sync();
  if (!cell_lu<G, double>(g, LU, N, w.piv, w.perm, w.invdiag)) return false;
  // the four stage increments
  for (int i = g.t; i < N; i += NT) w.u[0][i] = w.f[i];
  g.sync();
  cell_solve(g, LU, N, w.perm, w.invdiag, w.u[0]);
  for (int i = g.t; i < N; i += NT) w.ys[i] = fma(c_a21, w.u[0][i], w.y[i]);
  g.sync();
  cell_rates(m, g, p, w.ys, w.f, ed, (double*)nullptr, false);
  for (int i = g.t; i < N; i += NT) w.u[1][i] = fma(c_c21 * invh, w.u[0][i], w.f[i]);
  g.sync();
  cell_solve(g, LU, N, w.perm, w.invdiag, w.u[1]);
  for (int i = g.t; i < N; i += NT) w.ys[i] = w.y[i] + c_a31 * w.u[0][i] + c_a32 * w.u[1][i];
  g.sync();
  cell_rates(m, g, p, w.ys, w.f, ed, (double*)nullptr, false);
  for (int i = g.t; i < N; i += NT) w.u[2][i] = w.f[i] + invh * (c_c31 * w.u[0][i] + c_c32 * w.u[1][i]);
  g.sync();
  cell_solve(g, LU, N, w.perm, w.invdiag, w.u[2]);
  for (int i = g.t; i < N; i += NT)
    w.u[3][i] = w.f[i] + invh * (c_c41 * w.u[0][i] + c_c42 * w.u[1][i] + c_c43 * w.u[2][i]);
  g.sync();
  cell_solve(g, LU, N, w.perm, w.invdiag, w.u[3]);
  // reverse sweep over the stages (w.v[i] holds ub_i, then v_i = W^-T ub_i)
  for (int i = g.t; i < N; i += NT) {
    const double l = w.lam[i];
    w.ybar[i] = l;
#pragma unroll
    for (int k = 0; k < 4; ++k) w.v[k][i] = c_m[k] * l;
  }
  g.sync();
  solve_t(g, w, N, w.v[3]);
  for (int i = g.t; i < N; i += NT) {
    const double x = invh * w.v[3][i];
    w.v[2][i] = fma(c_c43, x, w.v[2][i]);
    w.v[1][i] = fma(c_c42, x, w.v[1][i]);
    w.v[0][i] = fma(c_c41, x, w.v[0][i]);
  }
  g.sync();
  solve_t(g, w, N, w.v[2]);
  // stages 3 and 4 share f(Y_3): J(Y_3)^T (v_3 + v_4) and the ln A terms with that weight
  for (int i = g.t; i < N; i += NT) {
    w.wv[i] = w.v[2][i] + w.v[3][i];
    w.ys[i] = w.y[i] + c_a31 * w.u[0][i] + c_a32 * w.u[1][i];
  }
  g.sync();
  {
    const CellScalars s3 = cell_rates<G, double, true>(m, g, p, w.ys, w.f, ed, scr, true, w.wv, Pd);
    cell_jacobian_vjp(m, g, s3, w.f, ed, scr, w.wv, abd, tzd, w.rhs);
  }
  for (int r = g.t; r < R; r += NT) w.gA[r] += Pd[r];
  for (int i = g.t; i < N; i += NT) {
    const double x = invh * w.v[2][i], r = w.rhs[i];
    w.v[1][i] += c_c32 * x + c_a32 * r;
    w.v[0][i] += c_c31 * x + c_a31 * r;
    w.ybar[i] += r;
  }
  g.sync();
  solve_t(g, w, N, w.v[1]);
  for (int i = g.t; i < N; i += NT) w.ys[i] = fma(c_a21, w.u[0][i], w.y[i]);
  g.sync();
  {
    const CellScalars s2 = cell_rates<G, double, true>(m, g, p, w.ys, w.f, ed, scr, true, w.v[1], Pd);
    cell_jacobian_vjp(m, g, s2, w.f, ed, scr, w.v[1], abd, tzd, w.rhs);
  }
  for (int r = g.t; r < R; r += NT) w.gA[r] += Pd[r];
  for (int i = g.t; i < N; i += NT) {
    const double r = w.rhs[i];
    w.v[0][i] += c_c21 * invh * w.v[1][i] + c_a21 * r;
    w.ybar[i] += r;
  }
  g.sync();
  solve_t(g, w, N, w.v[0]);
  // derivatives of J^T v_i and of v_i . df/dlnA along u_i at y (dual numbers): the derivative
  // parts are the terms of W's dependence on y; the value part of the first pass is
  // J(y)^T v_1 and v_1 . df/dlnA(y), the stage-1 terms
  Dual* scrD = reinterpret_cast<Dual*>(w.M);
  for (int k = 0; k < 4; ++k) {
    const double* uk = w.u[0] + k * w.n2;
    const double* vk = w.v[0] + k * w.n2;
    for (int i = g.t; i < N; i += NT) w.yd[i] = Dual(w.y[i], uk[i]);
    g.sync();
    const CellScalarsT<Dual> sd = cell_rates<G, Dual, true>(m, g, p, w.yd, w.fd, eD, scrD, true, vk, PD);
    cell_jacobian_vjp(m, g, sd, w.fd, eD, scrD, vk, abD, tzD, w.od);
    for (int i = g.t; i < N; i += NT) w.ybar[i] += (k == 0) ? w.od[i].v + w.od[i].d : w.od[i].d;
    for (int r = g.t; r < R; r += NT) w.gA[r] += (k == 0) ? PD[r].v + PD[r].d : PD[r].d;
    g.sync();
  }
  for (int i = g.t; i < N; i += NT) w.lam[i] = w.ybar[i];
  g.sync();
  return true;
}

struct AdjArgs {
  double p;
  const double* rec;
  int rec_cap;
  const int32_t* nsteps;
  const int32_t* status;
  const double *gT, *gY;
  double *gT0, *gY0;
  double* gcell;  // [ncells][R], file order
  int64_t ncells;
  int* queue;
  int* nfail;
};

template <int G>
__global__ void __launch_bounds__(256, 1) adjoint_kernel(DevMech m, AdjPlan plan, AdjArgs a) {
  extern __shared__ __align__(16) double smem[];
  constexpr int NT = Grp<G>::NT;
  Grp<G> g;
  g.init(threadIdx.x % NT, threadIdx.x / NT);
  double* base = smem + (size_t)g.gid * plan.total;
  const AdjMem w = carve_adj(base, plan);
  g.red = w.red;
  const EvalMem<double> ed = adj_eval_mem<double>(base, plan);
  const EvalMem<Dual> eD = adj_eval_mem<Dual>(base, plan);
  double* Pd = base + plan.off_P;
  Dual* PD = reinterpret_cast<Dual*>(base + plan.off_P);
  double* abd = base + plan.off_ab;
  Dual* abD = reinterpret_cast<Dual*>(abd);
  double* tzd = base + plan.off_tz;
  Dual* tzD = reinterpret_cast<Dual*>(tzd);
  const int N = m.N, K = m.K, R = m.R;
  const int64_t nc = a.ncells;
  for (;;) {
    if (g.t == 0) *w.slot = atomicAdd(a.queue, 1);
    g.sync();
    const int64_t cell = *w.slot;
    g.sync();
    if (cell >= nc) break;
    const int ns = a.nsteps[cell];
    bool ok = a.status[cell] == CHEM_CELL_OK && ns >= 0 && ns <= a.rec_cap;
    // dL/dphi at dt: Y_K(dt) = 1 - sum_{k<K} Y_k(dt)
    for (int i = g.t; i < N; i += NT)
      w.lam[i] = (i == 0) ? a.gT[cell] : a.gY[(size_t)(i - 1) * nc + cell] - a.gY[(size_t)(K - 1) * nc + cell];
    for (int r = g.t; r < R; r += NT) w.gA[r] = 0.0;
    g.sync();
    for (int n = ok ? ns - 1 : -1; n >= 0; --n) {
      const double* ck = a.rec + ((size_t)cell * a.rec_cap + n) * (N + 1);
      for (int i = g.t; i < N; i += NT) w.y[i] = ck[i];
      const double h = ck[N];
      g.sync();
      if (!adjoint_step(m, g, plan, a.p, h, w, ed, eD, abd, abD, tzd, tzD, Pd, PD)) {
        ok = false;
        if (g.t == 0) atomicAdd(a.nfail, 1);
        break;
      }
    }
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    for (int i = g.t; i < N; i += NT) {
      const double v = ok ? w.lam[i] : nan;
      if (i == 0) a.gT0[cell] = v;
      else a.gY0[(size_t)(i - 1) * nc + cell] = v;
    }
    if (g.t == 0) a.gY0[(size_t)(K - 1) * nc + cell] = ok ? 0.0 : nan;
    for (int r = g.t; r < R; r += NT) a.gcell[(size_t)cell * R + m.order[r]] = ok ? w.gA[r] : nan;
    g.sync();
  }
}

// g_lnA[r] = sum over cells of gcell[c][r] in a fixed order: partial sums over chunks of cells
// (one thread per reaction and chunk), then over the chunks.
__global__ void sum_chunks_kernel(const double* gcell, int64_t ncells, int R, int64_t chunk, double* partial) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = min(c0 + chunk, ncells);
  double s = 0.0;
  for (int64_t c = c0; c < c1; ++c) s += gcell[(size_t)c * R + r];
  partial[(size_t)blockIdx.y * R + r] = s;
}

__global__ void sum_partials_kernel(const double* partial, int nchunks, int R, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  double s = 0.0;
  for (int k = 0; k < nchunks; ++k) s += partial[(size_t)k * R + r];
  out[r] = s;
}

int64_t chunk_cells(int64_t ncells) { return std::max<int64_t>(256, (ncells + 65534) / 65535); }

}  // namespace

namespace chemgpu {

size_t adjoint_workspace_doubles(int R, int64_t ncells, bool have_cell_grads) {
  const int64_t nchunks = (ncells + chunk_cells(ncells) - 1) / chunk_cells(ncells);
  return (have_cell_grads ? 0 : (size_t)ncells * R) + (size_t)std::max<int64_t>(nchunks, 1) * R;
}

int adjoint_enqueue(const DevMech& d, int num_sms, size_t max_smem, double p_cgs, int64_t ncells, const double* rec,
                    int rec_cap, const int32_t* nsteps, const int32_t* status, const double* gT, const double* gY,
                    double* gT0, double* gY0, double* g_lnA, double* g_lnA_cells, double* ws, int* counters,
                    cudaStream_t st, std::string& err) {
  // launch shape: 8 warps per CTA; two cells of 4 warps when both working sets fit, else one
  // cell of 8 warps
  int G = 4, cpc = 2;
  AdjPlan plan = make_adj_plan(d.K, d.R, d.n_pd, d.n_pairs, G);
  if ((size_t)plan.total * sizeof(double) * cpc > max_smem) {
    G = 8;
    cpc = 1;
    plan = make_adj_plan(d.K, d.R, d.n_pd, d.n_pairs, G);
  }
  const size_t smem = (size_t)plan.total * sizeof(double) * cpc;
  if (smem > max_smem) {
    err = "chem_adjoint: working set of one cell (" + std::to_string(smem) + " B) exceeds a CTA's shared memory";
    return CHEM_ESIZE;
  }
  auto fail = [&](cudaError_t e, const char* what) {
    err = std::string("chem_adjoint: ") + what + ": " + cudaGetErrorString(e);
    return CHEM_ECUDA;
  };
  cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync");
  const void* fn = G == 4 ? (const void*)adjoint_kernel<4> : (const void*)adjoint_kernel<8>;
  const int threads = 32 * G * cpc;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return fail(e, "cudaFuncSetAttribute");
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
  if (e != cudaSuccess) return fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (occ < 1) {
    err = "chem_adjoint: kernel cannot be resident with its shared memory";
    return CHEM_ESIZE;
  }
  double* gcell = g_lnA_cells ? g_lnA_cells : ws;
  double* partial = g_lnA_cells ? ws : ws + (size_t)ncells * d.R;
  AdjArgs a;
  a.p = p_cgs; a.rec = rec; a.rec_cap = rec_cap; a.nsteps = nsteps; a.status = status;
  a.gT = gT; a.gY = gY; a.gT0 = gT0; a.gY0 = gY0; a.gcell = gcell; a.ncells = ncells;
  a.queue = counters; a.nfail = counters + 1;
  const int64_t ctas = (ncells + cpc - 1) / cpc;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)num_sms * occ));
  if (G == 4) adjoint_kernel<4><<<grid, threads, smem, st>>>(d, plan, a);
  else adjoint_kernel<8><<<grid, threads, smem, st>>>(d, plan, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "adjoint kernel launch");
  if (g_lnA) {
    const int64_t chunk = chunk_cells(ncells);
    const int nchunks = (int)((ncells + chunk - 1) / chunk);
    dim3 grid1((d.R + 127) / 128, nchunks);
    sum_chunks_kernel<<<grid1, 128, 0, st>>>(gcell, ncells, d.R, chunk, partial);
    sum_partials_kernel<<<(d.R + 127) / 128, 128, 0, st>>>(partial, nchunks, d.R, g_lnA);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "reduction kernel launch");
  }
  return CHEM_OK;
}

}  // namespace chemgpu
