// chemgpu host side and C ABI (see include/chemgpu.h): mechanism upload, launch shapes, CUDA
// graphs, the one-shot rate and Jacobian kernels, the mapping kernels and the probes.  The
// integrate kernels themselves are in integrate_device.cuh, compiled once per cell-group width
// (integrate_g*.cu).
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
#include "integrate.h"

namespace {
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

#ifdef CHEM_PHASE_TIMERS
// Per-phase cycle counters of the timer build; the integrate kernels add to them through
// IntegrateArgs::phase.
__device__ unsigned long long g_phase_cycles[8];
#endif

// Diagnostic: one cell group of 2 warps factors one matrix per CTA (chem_debug_lu).
__device__ inline void to_factor(double v, double& o) { o = v; }
__device__ inline void to_factor(double v, float& o) { o = __double2float_rn(v); }
__device__ inline void to_factor(double v, FF& o) { o = FF(v); }

__host__ __device__ inline int lu_probe_doubles(int N, int bytes) {
  return (N * N * bytes + 7) / 8 + (N * bytes + 7) / 8 + 12 + (2 * (N + 2) + 1) / 2;
}

template <typename S>
__global__ void __launch_bounds__(64) lu_probe_kernel(const double* A, int N, int64_t n, int variant, S* F, S* D,
                                                      int32_t* P, int32_t* sing) {
  extern __shared__ double smem[];
  Grp<2> g;
  g.init(threadIdx.x, 0);
  S* a = reinterpret_cast<S*>(smem);
  S* invd = reinterpret_cast<S*>(smem + (N * N * (int)sizeof(S) + 7) / 8);
  double* red = smem + (N * N * (int)sizeof(S) + 7) / 8 + (N * (int)sizeof(S) + 7) / 8;
  int* piv = reinterpret_cast<int*>(red + 12);
  int* perm = piv + N + 2;
  g.red = red;
  for (int64_t m = blockIdx.x; m < n; m += gridDim.x) {
    const double* Am = A + (size_t)m * N * N;
    for (int e = g.t; e < N * N; e += 64) to_factor(Am[e], a[e]);
    g.sync();
    const bool ok = cell_lu_any<2, S>(g, a, N, piv, perm, invd, variant);
    for (int e = g.t; e < N * N; e += 64) F[(size_t)m * N * N + e] = a[e];
    for (int i = g.t; i < N; i += 64) {
      D[(size_t)m * N + i] = invd[i];
      P[(size_t)m * N + i] = perm[i];
    }
    if (g.t == 0) sing[m] = ok ? 0 : 1;
    g.sync();
  }
}

__global__ void exp_probe_kernel(const double* x, double* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = exp_fast(x[i]);
}

}  // namespace

// ==========================================================================================
// Host side

namespace chemgpu {

const void* integrate_kernel_fn(int G, int solver) {
  switch (G) {
    case 1: return integrate_kernel_fn_g1(solver);
    case 2: return integrate_kernel_fn_g2(solver);
    case 4: return integrate_kernel_fn_g4(solver);
    case 8: return integrate_kernel_fn_g8(solver);
    default: return nullptr;
  }
}

void integrate_launch(int G, int solver, int grid, int threads, size_t smem, cudaStream_t st, const DevMech& d,
                      const IntegrateArgs& a) {
  switch (G) {
    case 1: integrate_launch_g1(solver, grid, threads, smem, st, d, a); break;
    case 2: integrate_launch_g2(solver, grid, threads, smem, st, d, a); break;
    case 4: integrate_launch_g4(solver, grid, threads, smem, st, d, a); break;
    default: integrate_launch_g8(solver, grid, threads, smem, st, d, a); break;
  }
}

}  // namespace chemgpu

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
  cudaEvent_t ev[2] = {nullptr, nullptr};  // brackets the integrate launches when stats are asked for
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

// Reaction split of cell_rates for a group of G warps.  The fall-off reactions come first in
// device order (Troe, then Lindemann), and a warp iteration that holds a Troe reaction costs about
// five plain ones (measured with clock64() per warp on the 53-species mechanism, evaluation with
// the Jacobian data: 34.7 k against 7.2 k cycles; four more exponentials, two logarithms and
// four Newton reciprocals), so interleaving the
// reactions over all warps leaves warp 0 with the slowest iterations while the others wait at the
// next barrier.  Warp 0 takes reactions [0, a) and the other G - 1 warps [a, R), with a a multiple
// of 32, at least the fall-off count, that minimises the larger side's cost (a warp iteration
// costing 5 with a Troe reaction, 2 with a Lindemann one, else 1).  If the plain interleaving
// (reaction r to thread r mod 32 G) costs no more, the split is 0, which keeps it.
#ifndef CHEM_TROE_ITER_COST
#define CHEM_TROE_ITER_COST 5
#endif
int reaction_split(int R, int n_troe, int n_fo, int G) {
  if (G <= 1) return R;
  auto iter_cost = [&](int s) { return (s < n_troe) ? CHEM_TROE_ITER_COST : (s < n_fo) ? 2 : 1; };
  int inter = 0;
  for (int w = 0; w < G; ++w) {
    int c = 0;
    for (int s = 32 * w; s < R; s += 32 * G) c += iter_cost(s);
    inter = std::max(inter, c);
  }
  const int top = (R + 31) / 32 * 32;
  int best_a = 0, best = inter;
  for (int a = 32; a <= top; a += 32) {
    if (a < n_fo) continue;
    int c0 = 0;
    for (int s = 0; s < a && s < R; s += 32) c0 += iter_cost(s);
    const int rest = std::max(0, R - a);
    const int c1 = (rest + 32 * (G - 1) - 1) / (32 * (G - 1));
    const int c = std::max(c0, c1);
    if (c < best) {
      best = c;
      best_a = std::min(a, R);
    }
  }
  return best_a;
}

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

#ifdef CHEM_PHASE_TIMERS
unsigned long long* phase_counters() {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_phase_cycles) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return static_cast<unsigned long long*>(p);
}
#endif

const void* integrate_fn(int G, int solver) { return integrate_kernel_fn(G, solver); }

const void* rates_fn(int G) {
  return G == 1 ? (const void*)rates_kernel<1>
         : G == 2 ? (const void*)rates_kernel<2>
         : G == 4 ? (const void*)rates_kernel<4>
                  : (const void*)rates_kernel<8>;
}

void launch_integrate(const Launch& L, cudaStream_t st, const DevMech& d, IntegrateArgs a) {
#ifdef CHEM_PHASE_TIMERS
  a.phase = phase_counters();
#endif
  integrate_launch(L.G, a.solver, L.grid, L.threads, L.smem, st, d, a);
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
  {
    int n_troe = 0;
    for (int r = 0; r < h.n_fo; ++r) n_troe += h.fo[(size_t)r * kFoDoubles + 7] != 0.0;
    d.rx_split[0] = h.R;
    for (int i = 1; i < 4; ++i) d.rx_split[i] = reaction_split(h.R, n_troe, h.n_fo, 1 << i);
  }
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
  for (cudaEvent_t e : m->ev)
    if (e) cudaEventDestroy(e);
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

int chem_mech_counts(const chem_mech* m, int* n_third_body, int* n_falloff) {
  if (!m) return set_err(CHEM_EINVAL, "chem_mech_counts: NULL mechanism");
  if (n_third_body) *n_third_body = m->host.n_tb;
  if (n_falloff) *n_falloff = m->host.n_fo;
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
  if (stats) {
    for (cudaEvent_t& e : m->ev)
      if (!e) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(m->ev[0], st));
  }
  if (o.use_graph) {
    rc = launch_via_graph(m, o, a, st);
  } else {
    rc = enqueue_integrate(m, o, a, st);
  }
  if (rc) return rc;
  if (stats) CK(cudaEventRecord(m->ev[1], st));
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
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, m->ev[0], m->ev[1]));
    stats->kernel_ms = ms;
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

int chem_debug_lu(const double* A, int N, int64_t n, int precision, int variant, void* factors, void* invdiag,
                  int32_t* perm, int32_t* singular, void* stream) {
  if (N < 1 || N > 128 || n < 0) return set_err(CHEM_EINVAL, "chem_debug_lu: need 1 <= N <= 128 and n >= 0");
  if (precision != CHEM_PREC_FP64 && precision != CHEM_PREC_MIXED && precision != CHEM_PREC_MIXED_FF)
    return set_err(CHEM_EINVAL, "chem_debug_lu: unknown precision");
  if (variant < 0 || variant > 2) return set_err(CHEM_EINVAL, "chem_debug_lu: variant must be 0, 1 or 2");
  if (n == 0) return CHEM_OK;
  if (!is_device_ptr(A) || !is_device_ptr(factors) || !is_device_ptr(invdiag) || !is_device_ptr(perm) ||
      !is_device_ptr(singular))
    return set_err(CHEM_EINVAL, "chem_debug_lu: device arrays only");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)std::min<int64_t>(n, 65535);
  const int bytes = precision == CHEM_PREC_MIXED ? 4 : 8;
  const size_t smem = sizeof(double) * (size_t)lu_probe_doubles(N, bytes);
  if (precision == CHEM_PREC_FP64) {
    CK(cudaFuncSetAttribute(lu_probe_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    lu_probe_kernel<double><<<grid, 64, smem, st>>>(A, N, n, variant, static_cast<double*>(factors),
                                                    static_cast<double*>(invdiag), perm, singular);
  } else if (precision == CHEM_PREC_MIXED) {
    CK(cudaFuncSetAttribute(lu_probe_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    lu_probe_kernel<float><<<grid, 64, smem, st>>>(A, N, n, variant, static_cast<float*>(factors),
                                                   static_cast<float*>(invdiag), perm, singular);
  } else {
    CK(cudaFuncSetAttribute(lu_probe_kernel<FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    lu_probe_kernel<FF><<<grid, 64, smem, st>>>(A, N, n, variant, static_cast<FF*>(factors),
                                                static_cast<FF*>(invdiag), perm, singular);
  }
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
