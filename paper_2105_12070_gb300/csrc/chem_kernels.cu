// chemgpu kernels and C ABI (see include/chemgpu.h).
//
// GPU design (GB300, sm_103a).  One warp integrates one cell at a time; a CTA holds several
// independent cell warps; a persistent grid pulls cells from a device work queue (one atomic
// per cell), so that cells of very different stiffness balance across SMs -- the on-device
// counterpart of the paper's MPI load balancing (Sec. 2.2).  Each warp keeps its cell's whole
// working set in shared memory: the dense Jacobian (Sec. 2.3), the iteration matrix and its LU
// factors, the stage vectors and the per-reaction scratch.
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
#include "chem_internal.h"

using namespace chemgpu;

namespace {

constexpr double kRu = 8.314462618e7;  // erg/(mol K)
constexpr double kPatm = 1.01325e6;    // dyn/cm^2
constexpr double kLnPatmRu = -4.4074185890025275;  // ln(Patm / Ru), Patm/Ru in mol K / cm^3
constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------------------------
// Rosenbrock method (transformed form of Hairer & Wanner IV.7): with W = I/(gamma h) - J,
//   W u_i = f(y + sum_j a_ij u_j) + sum_j (c_ij / h) u_j,  y_new = y + sum m_i u_i,
//   error = sum e_i u_i.  4 stages, order 4(3), L-stable; a_4j = a_3j so stage 4 reuses the
// rate evaluation of stage 3.  (gamma is the root near 0.5728 of the order-4 L-stability
// polynomial; the classical coefficients alpha_21 = 2 gamma, alpha_3 = 0.65, b_3 = 0,
// beta_43 = -0.23 and R_hat(inf) = 1/2 fix the rest through the order conditions.)
__constant__ double c_gamma = 0.5728160624821348554080014;
__constant__ double c_a21 = 2.0;
__constant__ double c_a31 = 1.860719413892191158443;
__constant__ double c_a32 = 0.2350527673509341985179;
__constant__ double c_c21 = -7.137649921358897064356;
__constant__ double c_c31 = 2.514641112124939467064;
__constant__ double c_c32 = 0.6358184234567149330241;
__constant__ double c_c41 = -2.12191165112287042299;
__constant__ double c_c42 = -0.3261607745737058543668;
__constant__ double c_c43 = -0.7009668191330486406986;
__constant__ double c_m[4] = {2.258943599044704060723, 0.294864173772259595933, 0.4414500735399588815281,
                              1.099433447424383102325};
__constant__ double c_e[4] = {-0.2561963508749719744122, -0.07156405471952786716643,
                              -0.09930846885424478507654, -0.9949360460805926517866};

// ------------------------------------------------------------------------------------------
// Cell groups.  G warps (32 G threads) cooperate on one cell; several groups share a CTA and
// synchronise with their own named barrier (ids 1..15).  Reductions go through a small
// per-group scratch in a fixed order, so results do not depend on scheduling.

template <int G>
struct Grp {
  static constexpr int NT = 32 * G;
  int t;        // thread index in the group
  int gid;      // group index in the CTA
  double* red;  // 6 G doubles of reduction scratch
  mutable int parity;

  __device__ int lane() const { return t & 31; }
  __device__ int warp() const { return t >> 5; }
  __device__ void sync() const {
    if (G == 1) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(NT) : "memory");
    }
  }
  __device__ double sum(double v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (G == 1) return v;
    double* r = red + (parity & 1) * 3 * G;  // alternate halves: no reader of the previous
    parity++;                                // call can still be reading this one
    if (lane() == 0) r[warp()] = v;
    sync();
    double s = r[0];
#pragma unroll
    for (int i = 1; i < G; ++i) s += r[i];
    return s;
  }
  // two sums at once (one exchange)
  __device__ void sum2(double& a, double& b) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
    }
    if (G == 1) return;
    double* r = red + (parity & 1) * 3 * G;
    parity++;
    if (lane() == 0) { r[2 * warp()] = a; r[2 * warp() + 1] = b; }
    sync();
    a = r[0];
    b = r[1];
#pragma unroll
    for (int i = 1; i < G; ++i) { a += r[2 * i]; b += r[2 * i + 1]; }
  }
  // max that propagates NaN (a NaN error norm must reject the step)
  __device__ static double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }
  __device__ double max_nan(double v) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
    if (G == 1) return v;
    double* r = red + (parity & 1) * 3 * G;
    parity++;
    if (lane() == 0) r[warp()] = v;
    sync();
    double s = r[0];
#pragma unroll
    for (int i = 1; i < G; ++i) s = nanmax(s, r[i]);
    return s;
  }
  // argmax of key (ties to the lowest index) over the group, carrying a value along
  __device__ void argmax(long long& key, int& idx, double& val) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ok = __shfl_xor_sync(kFull, key, o);
      const int oi = __shfl_xor_sync(kFull, idx, o);
      const double ov = __shfl_xor_sync(kFull, val, o);
      if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; val = ov; }
    }
    if (G == 1) return;
    double* r = red + (parity & 1) * 3 * G;
    parity++;
    if (lane() == 0) {
      r[3 * warp()] = __longlong_as_double(key);
      r[3 * warp() + 1] = __int2double_rn(idx);
      r[3 * warp() + 2] = val;
    }
    sync();
    key = __double_as_longlong(r[0]);
    idx = (int)r[1];
    val = r[2];
#pragma unroll
    for (int i = 1; i < G; ++i) {
      const long long ok = __double_as_longlong(r[3 * i]);
      const int oi = (int)r[3 * i + 1];
      if (ok > key || (ok == key && oi < idx)) { key = ok; idx = oi; val = r[3 * i + 2]; }
    }
  }
};

// ------------------------------------------------------------------------------------------
// Per-cell shared-memory plan (doubles).

struct Plan {
  int N, K, R, n_pd, G;
  int SA;  // size of each of the two matrix buffers: max(N*N, 8*R)
  int off_A, off_B, off_vec, off_sp, off_q, off_M, off_piv, off_red, total;
};

__host__ __device__ inline int round2(int x) { return (x + 1) & ~1; }

__host__ __device__ inline Plan make_plan(int K, int R, int n_pd, int G) {
  Plan p;
  p.N = K; p.K = K; p.R = R; p.n_pd = n_pd; p.G = G;
  p.SA = round2(max(K * K, 8 * R));
  p.off_A = 0;
  p.off_B = p.SA;
  p.off_vec = 2 * p.SA;
  // vectors: y, ynew, f0, fs, u0..u3, err, invdiag, rhs, res, (er, ec as ints), (FP32 inverse
  // pivots)  (14 x N); the Jacobian's temporaries zc, dwT, rowA, rowB, ccol reuse u0..u3, err
  p.off_sp = p.off_vec + 14 * round2(K);
  // species: C, hRT, cpR, gRT, omega, dcpR  (6 x K)
  p.off_q = p.off_sp + 6 * round2(K);
  p.off_M = p.off_q + round2(R);
  p.off_piv = p.off_M + round2(max(n_pd, 1));
  p.off_red = p.off_piv + round2(K + 2);  // pivots and the composed permutation (ints)
  p.total = p.off_red + 6 * G + 2;  // reduction scratch + queue slot
  p.total = round2(p.total);
  return p;
}

struct CellMem {
  double *A, *B;
  double *y, *ynew, *f0, *fs, *u[4], *err, *invdiag, *zc, *dwT, *rowA, *rowB, *ccol, *rhs, *res;
  int *er, *ec;
  float* invd32;
  double *C, *hRT, *cpR, *gRT, *omega, *dcpR;
  double *q, *M, *red;
  int* piv;
  int* perm;
  int* slot;
};

__device__ inline CellMem carve(double* base, const Plan& p) {
  CellMem w;
  w.A = base + p.off_A;
  w.B = base + p.off_B;
  const int n = round2(p.K);
  double* v = base + p.off_vec;
  w.y = v; w.ynew = v + n; w.f0 = v + 2 * n; w.fs = v + 3 * n;
  for (int i = 0; i < 4; ++i) w.u[i] = v + (4 + i) * n;
  w.err = v + 8 * n; w.invdiag = v + 9 * n;
  w.zc = w.u[0]; w.dwT = w.u[1]; w.rowA = w.u[2]; w.rowB = w.u[3]; w.ccol = w.err;
  w.rhs = v + 10 * n; w.res = v + 11 * n;
  w.er = reinterpret_cast<int*>(v + 12 * n);
  w.ec = w.er + n;
  w.invd32 = reinterpret_cast<float*>(v + 13 * n);
  double* s = base + p.off_sp;
  w.C = s; w.hRT = s + n; w.cpR = s + 2 * n; w.gRT = s + 3 * n; w.omega = s + 4 * n; w.dcpR = s + 5 * n;
  w.q = base + p.off_q;
  w.M = base + p.off_M;
  w.piv = reinterpret_cast<int*>(base + p.off_piv);
  w.perm = w.piv + p.K + 2;
  w.red = base + p.off_red;
  w.slot = reinterpret_cast<int*>(base + p.off_red + 6 * p.G);
  return w;
}

// ------------------------------------------------------------------------------------------
// Thermochemistry and rates (Eq. 1).  Scalars of the cell state, identical in every thread.

struct CellScalars {
  double T, invT, lnT, rho, inv_rho, Wbar, cp, dcp_dT, fT;
};

// exp(x) for the rate constants: Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic", ACM TOMS 15,
// 1989): x = (32 m + j) ln2/32 + r with |r| <= ln2/64, exp(x) = 2^m 2^(j/32) (1 + p(r)), p the
// degree-6 Taylor polynomial (truncation below 2e-18), 2^(j/32) as a double-double.  About 12
// FP64 operations instead of a library call's ~17; |x| >= 708 and NaN go to exp().
__device__ const double c_exp2_j32[64] = {
    0x1.0000000000000p+0, 0x0.0p+0,
    0x1.059b0d3158574p+0, 0x1.d73e2a475b465p-55,
    0x1.0b5586cf9890fp+0, 0x1.8a62e4adc610bp-54,
    0x1.11301d0125b51p+0, -0x1.6c51039449b3ap-54,
    0x1.172b83c7d517bp+0, -0x1.19041b9d78a76p-55,
    0x1.1d4873168b9aap+0, 0x1.e016e00a2643cp-54,
    0x1.2387a6e756238p+0, 0x1.9b07eb6c70573p-54,
    0x1.29e9df51fdee1p+0, 0x1.612e8afad1255p-55,
    0x1.306fe0a31b715p+0, 0x1.6f46ad23182e4p-55,
    0x1.371a7373aa9cbp+0, -0x1.63aeabf42eae2p-54,
    0x1.3dea64c123422p+0, 0x1.ada0911f09ebcp-55,
    0x1.44e086061892dp+0, 0x1.89b7a04ef80d0p-59,
    0x1.4bfdad5362a27p+0, 0x1.d4397afec42e2p-56,
    0x1.5342b569d4f82p+0, -0x1.07abe1db13cadp-55,
    0x1.5ab07dd485429p+0, 0x1.6324c054647adp-54,
    0x1.6247eb03a5585p+0, -0x1.383c17e40b497p-54,
    0x1.6a09e667f3bcdp+0, -0x1.bdd3413b26456p-54,
    0x1.71f75e8ec5f74p+0, -0x1.16e4786887a99p-55,
    0x1.7a11473eb0187p+0, -0x1.41577ee04992fp-55,
    0x1.82589994cce13p+0, -0x1.d4c1dd41532d8p-54,
    0x1.8ace5422aa0dbp+0, 0x1.6e9f156864b27p-54,
    0x1.93737b0cdc5e5p+0, -0x1.75fc781b57ebcp-57,
    0x1.9c49182a3f090p+0, 0x1.c7c46b071f2bep-56,
    0x1.a5503b23e255dp+0, -0x1.d2f6edb8d41e1p-54,
    0x1.ae89f995ad3adp+0, 0x1.7a1cd345dcc81p-54,
    0x1.b7f76f2fb5e47p+0, -0x1.5584f7e54ac3bp-56,
    0x1.c199bdd85529cp+0, 0x1.11065895048ddp-55,
    0x1.cb720dcef9069p+0, 0x1.503cbd1e949dbp-56,
    0x1.d5818dcfba487p+0, 0x1.2ed02d75b3707p-55,
    0x1.dfc97337b9b5fp+0, -0x1.1a5cd4f184b5cp-54,
    0x1.ea4afa2a490dap+0, -0x1.e9c23179c2893p-54,
    0x1.f50765b6e4540p+0, 0x1.9d3e12dd8a18bp-54};

__device__ inline double exp_fast(double x) {
  if (!(fabs(x) < 708.0)) return exp(x);
  const double shifter = 0x1.8p52;  // adding it rounds x 32/ln2 to an integer in the low bits
  const double t = fma(x, 0x1.71547652b82fep+5, shifter);
  const int k = (int)__double2loint(t);
  const double kd = t - shifter;
  double r = fma(-kd, 0x1.62e42fefa39efp-6, x);  // ln2/32, high part
  r = fma(-kd, 0x1.abc9e3b39803fp-61, r);        // ln2/32, low part
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(r, q, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const int j = k & 31;
  const double th = __ldg(&c_exp2_j32[2 * j]), tl = __ldg(&c_exp2_j32[2 * j + 1]);
  const double res = fma(th, p, tl) + th;
  // times 2^(k >> 5): add to the exponent field (the result stays normal for |x| < 708)
  return __longlong_as_double(__double_as_longlong(res) + ((long long)(k >> 5) << 52));
}

// 2^k as a double (|k| < 1000), exact.
__device__ inline double pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Binary exponent of |a| (the biased exponent field; 0 for zero and subnormals).
__device__ inline int exp_field(double a) { return (int)((__double_as_longlong(a) >> 52) & 0x7ff); }

// NASA-7: cp/R, h/RT, s/R and d(cp/R)/dT.
__device__ inline void nasa7(const double* a, double T, double invT, double lnT, double& cpR, double& hRT,
                             double& sR, double& dcpR) {
  cpR = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  hRT = a[0] + T * (a[1] * 0.5 + T * (a[2] * (1.0 / 3.0) + T * (a[3] * 0.25 + T * a[4] * 0.2))) + a[5] * invT;
  sR = a[0] * lnT + T * (a[1] + T * (a[2] * 0.5 + T * (a[3] * (1.0 / 3.0) + T * a[4] * 0.25))) + a[6];
  dcpR = a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]));
}

// Troe broadening: F and d log10 F / d log10 Pr; with jac also d ln F / dT at fixed Pr.
__device__ inline void troe(const double* fo, double T, double invT, double Pr, double& F, double& dlF,
                            double& dlnF_dT, bool jac) {
  const double a = fo[3], T3 = fo[4], T1 = fo[5], T2 = fo[6];
  const double e3 = exp_fast(-T / T3), e1 = exp_fast(-T / T1), e2 = exp_fast(-T2 * invT);
  const double Fcent = (1.0 - a) * e3 + a * e1 + e2;
  const double L = log10(Fcent);
  const double c = -0.4 - 0.67 * L, n = 0.75 - 1.27 * L;
  const double x = log10(Pr);
  const double den = n - 0.14 * (x + c);
  const double f1 = (x + c) / den;
  const double g = 1.0 + f1 * f1;
  F = exp_fast(2.302585092994045684 * (L / g));
  dlF = -2.0 * L * f1 / (g * g) * (n / (den * den));
  dlnF_dT = 0.0;
  if (jac) {
    const double dFc = -(1.0 - a) / T3 * e3 - a / T1 * e1 + T2 * invT * invT * e2;
    const double dL = dFc / (Fcent * 2.302585092994045684);
    const double df1_dL = (-0.67 * den - (x + c) * (-1.27 + 0.14 * 0.67)) / (den * den);
    const double dlog10F_dL = 1.0 / g - L * 2.0 * f1 / (g * g) * df1_dL;
    dlnF_dT = 2.302585092994045684 * dlog10F_dL * dL;
  }
}

// Evaluates f(y) into f[0..N).  With jac, also leaves per-reaction derivative data in
// scr[r*8 + 0..7] = {dq/dC at the 4 distinct slot species, phi (coefficient of the
// efficiencies), sum_j dq/dC_j C_j, dq/dT at fixed C, reaction enthalpy (erg/mol)} and the
// species production rates in w.omega.
template <int G>
__device__ CellScalars cell_rates(const DevMech& m, const Grp<G>& g, double p, const double* y, double* f,
                                  const CellMem& w, double* scr, bool jac) {
  constexpr int NT = Grp<G>::NT;
  const int K = m.K, d = K - 1;
  CellScalars s;
  s.T = y[0];
  s.invT = 1.0 / s.T;
  s.lnT = log(s.T);
  // mass fractions, mean molar mass, density, concentrations, thermo
  double ysum = 0.0, yw = 0.0;
  for (int k = g.t; k < d; k += NT) {
    const double Yk = y[1 + k];
    ysum += Yk;
    yw += Yk * m.sp[k * kSpDoubles + 1];
  }
  g.sum2(ysum, yw);
  const double Yd = 1.0 - ysum;
  yw += Yd * m.sp[d * kSpDoubles + 1];
  s.Wbar = 1.0 / yw;
  s.rho = p * s.Wbar / (kRu * s.T);
  s.inv_rho = yw * kRu * s.T / p;
  double cp = 0.0, dcp = 0.0;
  for (int k = g.t; k < K; k += NT) {
    const double* sp = m.sp + k * kSpDoubles;
    const double Yk = (k < d) ? y[1 + k] : Yd;
    w.C[k] = s.rho * Yk * sp[1];
    const double* a = (s.T <= sp[2]) ? sp + 3 : sp + 10;
    double cpR, hRT, sR, dcpR;
    nasa7(a, s.T, s.invT, s.lnT, cpR, hRT, sR, dcpR);
    w.cpR[k] = cpR;
    w.hRT[k] = hRT;
    w.gRT[k] = hRT - sR;
    w.dcpR[k] = dcpR;
    cp += Yk * cpR * sp[1];
    dcp += Yk * dcpR * sp[1];
  }
  g.sum2(cp, dcp);
  s.cp = cp * kRu;
  s.dcp_dT = dcp * kRu;
  g.sync();
  // third-body concentrations [M]_r = sum_k eff_rk C_k of the pressure-dependent reactions
  for (int r = g.t; r < m.n_pd; r += NT) {
    const double* e = m.eff + (size_t)r * K;
    double a0 = 0.0, a1 = 0.0;
    int k = 0;
    for (; k + 1 < K; k += 2) {
      a0 = fma(e[k], w.C[k], a0);
      a1 = fma(e[k + 1], w.C[k + 1], a1);
    }
    if (k < K) a0 = fma(e[k], w.C[k], a0);
    w.M[r] = a0 + a1;
  }
  g.sync();
  const double ln_patm_rut = kLnPatmRu - s.lnT;  // ln(Patm / (Ru T))
  for (int r = g.t; r < m.R; r += NT) {
    const int* ii = m.rxi + r * kRxInts;
    const double* rd = m.rxd + r * kRxDoubles;
    const int a0 = ii[0], a1 = ii[1], p0 = ii[2], p1 = ii[3];
    const double Ca0 = w.C[a0], Ca1 = (a1 >= 0) ? w.C[a1] : 1.0;
    const double Cp0 = w.C[p0], Cp1 = (p1 >= 0) ? w.C[p1] : 1.0;
    const double pf = Ca0 * Ca1, pr = Cp0 * Cp1;
    double kf = exp_fast(fma(rd[1], s.lnT, rd[0]) - rd[2] * s.invT);
    double dG = w.gRT[p0] - w.gRT[a0];
    if (p1 >= 0) dG += w.gRT[p1];
    if (a1 >= 0) dG -= w.gRT[a1];
    const int dnu = m.dnu[r];
    // 1/Kc = exp(sum nu g/RT - dnu ln(Patm/(Ru T)))
    const double invKc = exp_fast(dG - dnu * ln_patm_rut);
    double mfac = 1.0, Mr = 0.0;
    double Pr = 0.0, F = 1.0, dlF = 0.0, dlnF_dT = 0.0, k0 = 0.0;
    const bool pd = r < m.n_pd;
    const bool fo = r < m.n_fo;
    const double* fop = nullptr;
    if (pd) Mr = w.M[r];
    if (fo) {
      fop = m.fo + (size_t)r * kFoDoubles;
      k0 = exp_fast(fma(fop[1], s.lnT, fop[0]) - fop[2] * s.invT);
      Pr = k0 * Mr / kf;
      if (fop[7] != 0.0) troe(fop, s.T, s.invT, Pr, F, dlF, dlnF_dT, jac);
      kf = kf * Pr / (1.0 + Pr) * F;
    } else if (pd) {
      mfac = Mr;
    }
    const double kr = kf * invKc;
    const double q = mfac * (kf * pf - kr * pr);
    w.q[r] = q;
    if (jac) {
      double* o = scr + (size_t)r * 8;
      double dH = w.hRT[p0] - w.hRT[a0];
      if (p1 >= 0) dH += w.hRT[p1];
      if (a1 >= 0) dH -= w.hRT[a1];
      const double dlnKc_dT = (dH - dnu) * s.invT;
      const double dlnkinf = (rd[1] + rd[2] * s.invT) * s.invT;
      double phi = 0.0, dlnk = dlnkinf;
      if (fo) {
        const double inv1p = 1.0 / (1.0 + Pr);
        const double dk_dM = k0 * F * inv1p * (inv1p + dlF);
        phi = dk_dM * (pf - invKc * pr);
        const double dlnk0 = (fop[1] + fop[2] * s.invT) * s.invT;
        dlnk = dlnkinf + (inv1p + dlF) * (dlnk0 - dlnkinf) + dlnF_dT;
      } else if (pd) {
        phi = kf * pf - kr * pr;
      }
      const double dqdT = mfac * (kf * dlnk * pf - kr * (dlnk - dlnKc_dT) * pr);
      double DC = phi * Mr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = ii[4 + u];
        double D = 0.0;
        if (j >= 0) {
          const double dpf = (a0 == j ? Ca1 : 0.0) + (a1 == j ? Ca0 : 0.0);
          const double dpr = (p0 == j ? Cp1 : 0.0) + (p1 == j ? Cp0 : 0.0);
          D = mfac * (kf * dpf - kr * dpr);
          DC = fma(D, w.C[j], DC);
        }
        o[u] = D;
      }
      o[4] = phi;
      o[5] = DC;
      o[6] = dqdT;
      o[7] = dH * kRu * s.T;
    }
  }
  g.sync();
  // species production rates and the source term
  double Qp = 0.0;
  for (int k = g.t; k < K; k += NT) {
    double om = 0.0;
    for (int e = m.sr_ptr[k]; e < m.sr_ptr[k + 1]; ++e) om = fma(m.sr_nu[e], w.q[m.sr_idx[e]], om);
    w.omega[k] = om;
    Qp = fma(w.hRT[k], om, Qp);
    if (k < d) f[1 + k] = m.sp[k * kSpDoubles] * om * s.inv_rho;
  }
  const double Q = g.sum(Qp) * kRu * s.T;
  s.fT = -Q * s.inv_rho / s.cp;
  if (g.t == 0) f[0] = s.fT;
  g.sync();
  return s;
}

// Assemble the analytical Jacobian (Sec. 2.3) at the state of the preceding cell_rates(jac)
// call.  J (overwritten) holds the per-reaction data on entry, Z is N*N scratch, J receives
// -d f / d phi (stored negated, so that W = I/(gamma h) - J is a copy plus the diagonal).  Chain rule through C_j = rho Y_j / W_j, rho = p Wbar/(Ru T), Y_K = 1 - sum Y_i;
// Z rows k < K-1 hold d omega_k / dC, row K-1 holds d Q / dC (Q = sum_k H_k omega_k).
template <int G>
__device__ void cell_jacobian(const DevMech& m, const Grp<G>& g, const CellScalars& s, const double* f,
                              const CellMem& w, double* J, double* Z) {
  constexpr int NT = Grp<G>::NT;
  const int K = m.K, N = K, d = K - 1;
  const double* scr = J;
  for (int e = g.t; e < N * N; e += NT) Z[e] = 0.0;
  g.sync();
  // mass-action part: one thread per receiving Z entry sums its contributions (a fixed plan
  // built with the mechanism; no two threads write the same entry, no atomics)
  for (int e = g.t; e < m.zg_entries; e += NT) {
    double acc = 0.0;
    const int cb = m.zg_ptr[e], ce = m.zg_ptr[e + 1];
    for (int c = cb; c < ce; ++c) acc = fma(m.zg_coef[c], scr[m.zg_src[c]], acc);
    Z[m.zg_dst[e]] = acc;
  }
  g.sync();
  // efficiency part of the pressure-dependent reactions: Z[k][j] += sum_r v_kr eff_rj over the
  // (row k, reaction r) pairs, v_kr = nu_kr phi_r.  The coefficients go to the stage-vector area
  // first (free while the Jacobian is built).
  double* v = w.u[0];
  for (int c = g.t; c < m.n_pairs; c += NT) v[c] = m.pr_nu[c] * scr[(size_t)m.pr_pd[c] * 8 + 4];
  g.sync();
  {
    const float invK = 1.0f / (float)K;
    const int items = m.n_prows * K;
    for (int x = g.t; x < items; x += NT) {
      const int ri = (int)(((float)x + 0.5f) * invK), j = x - ri * K;
      const int row = m.pr_rows[ri];
      double acc = 0.0;
      for (int c = m.pr_ptr[row]; c < m.pr_ptr[row + 1]; ++c) acc = fma(v[c], m.eff[(size_t)m.pr_pd[c] * K + j], acc);
      Z[row * N + j] += acc;
    }
  }
  g.sync();
  // per-species gathers of sum_j dq/dC_j C_j and dq/dT; enthalpy weights of the species rows
  const double invWd = m.sp[d * kSpDoubles + 1];
  const double RuT = kRu * s.T;
  double* wq = w.res;
  for (int k = g.t; k < d; k += NT) {
    double zc = 0.0, dw = 0.0;
    for (int e = m.sr_ptr[k]; e < m.sr_ptr[k + 1]; ++e) {
      const double nu = m.sr_nu[e];
      const int r = m.sr_idx[e];
      zc = fma(nu, scr[(size_t)r * 8 + 5], zc);
      dw = fma(nu, scr[(size_t)r * 8 + 6], dw);
    }
    w.zc[k] = zc;
    w.dwT[k] = dw;
    // mass conservation (sum_k W_k omega_k = 0) gives omega_K = -sum_{k<K} (W_k/W_K) omega_k, so
    // Q = sum_k H_k omega_k = sum_{k<K} (H_k - H_K W_k/W_K) omega_k: the enthalpy row is a
    // weighted sum of the species rows
    wq[k] = RuT * (w.hRT[k] - w.hRT[d] * m.sp[k * kSpDoubles] * invWd);
  }
  g.sync();
  // enthalpy row Z_Q[j] = sum_k wq_k Z[k][j] (stored in row K-1), with sum_j Z_Q[j] C_j and
  // dQ/dT|_C = sum_k wq_k dw_k/dT|_C
  double zqc = 0.0, dqt = 0.0, cpw = 0.0;
  for (int j = g.t; j < K; j += NT) {
    double a0 = 0.0, a1 = 0.0;
    int k = 0;
    for (; k + 1 < d; k += 2) {
      a0 = fma(wq[k], Z[k * N + j], a0);
      a1 = fma(wq[k + 1], Z[(k + 1) * N + j], a1);
    }
    if (k < d) a0 = fma(wq[k], Z[k * N + j], a0);
    const double zq = a0 + a1;
    Z[d * N + j] = zq;
    zqc = fma(zq, w.C[j], zqc);
    cpw = fma(w.cpR[j], w.omega[j], cpw);
  }
  for (int k = g.t; k < d; k += NT) dqt = fma(wq[k], w.dwT[k], dqt);
  g.sum2(zqc, dqt);
  cpw = g.sum(cpw) * kRu;
  g.sync();
  // per-row and per-column factors
  for (int k = g.t; k < d; k += NT) {
    const double Wk = m.sp[k * kSpDoubles];
    w.rowA[k] = Wk * invWd * Z[k * N + d];
    w.rowB[k] = Wk * s.inv_rho * (w.zc[k] - w.omega[k]);
    w.ccol[k] = -s.Wbar * (m.sp[k * kSpDoubles + 1] - invWd);
  }
  g.sync();
  const double inv_rhocp = s.inv_rho / s.cp;
  const double inv_cp = 1.0 / s.cp;
  const double fT = s.fT;
  // temperature row and column, then the species block (J now overwrites the scratch)
  const double ZQd = Z[d * N + d];
  const double cpd = w.cpR[d] * invWd;
  for (int i = g.t; i < d; i += NT) {
    const double ci = w.ccol[i];
    const double invWi = m.sp[i * kSpDoubles + 1];
    const double dQdY = s.rho * (invWi * Z[d * N + i] - invWd * ZQd) + zqc * ci;
    const double dcpdY = (w.cpR[i] * invWi - cpd) * kRu;
    J[1 + i] = fma(dQdY, inv_rhocp, fT * (ci + dcpdY * inv_cp));
    const double Wk = m.sp[i * kSpDoubles];
    J[(1 + i) * N] = -(Wk * s.inv_rho * (w.dwT[i] - w.zc[i] * s.invT) + f[1 + i] * s.invT);
  }
  if (g.t == 0) J[0] = (cpw + dqt - zqc * s.invT) * inv_rhocp + fT * (-s.invT + s.dcp_dT * inv_cp);
  const int nb = d * d;
  const float inv_d = 1.0f / (float)d;
  for (int e = g.t; e < nb; e += NT) {
    const int k = (int)(((float)e + 0.5f) * inv_d), i = e - k * d;
    const double Wk = m.sp[k * kSpDoubles];
    const double invWi = m.sp[i * kSpDoubles + 1];
    J[(1 + k) * N + 1 + i] = fma(-w.rowB[k], w.ccol[i], fma(-Wk * invWi, Z[k * N + i], w.rowA[k]));
  }
  g.sync();
}

// ------------------------------------------------------------------------------------------
// Dense LU with partial pivoting (row interchanges, ties to the lowest row), in place, and the
// substitutions that use it (Sec. 2.3: dense LU + back substitution).  Returns false on an
// exactly zero pivot.

// |a| as an ordered integer key (bit pattern of a non-negative float / double)
__device__ inline long long abs_key(double a) { return __double_as_longlong(fabs(a)); }
__device__ inline long long abs_key(float a) { return (long long)__float_as_int(fabsf(a)); }

template <int G, typename S>
__device__ bool cell_lu(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag) {
  constexpr int NT = Grp<G>::NT;
  bool ok = true;
  for (int k = 0; k < N; ++k) {
    // pivot: largest |a_ik|, compared as the bit patterns of |a| (monotone for non-negative)
    long long best = -1;
    int bi = N;
    double bv = 0.0;
    for (int i = k + g.t; i < N; i += NT) {
      const S a = A[i * N + k];
      const long long v = abs_key(a);
      if (v > best) { best = v; bi = i; bv = (double)a; }
    }
    g.argmax(best, bi, bv);
    // one thread takes the reciprocal of the pivot while the others swap the rows
    if (g.t == 0) {
      piv[k] = bi;
      invdiag[k] = S(1) / S(bv);
    }
    if (best <= 0) ok = false;  // zero column: singular
    if (bi != k) {
      for (int j = g.t; j < N; j += NT) {
        const S t = A[k * N + j];
        A[k * N + j] = A[bi * N + j];
        A[bi * N + j] = t;
      }
    }
    g.sync();
    const S inv = invdiag[k];
    for (int i = k + 1 + g.t; i < N; i += NT) A[i * N + k] *= inv;
    g.sync();
    const int mm = N - k - 1;
    const int tot = mm * mm;
    if (tot > 0) {
      const float inv_m = 1.0f / (float)mm;
      S* Ak = A + (size_t)(k + 1) * N + k;  // column k of the trailing rows
      const S* U = A + (size_t)k * N + k + 1;  // pivot row right of the diagonal
      S* T0 = A + (size_t)(k + 1) * N + k + 1;
      // four independent updates per thread and iteration (loads first, then the FMAs)
      int e = g.t;
      for (; e + 3 * NT < tot; e += 4 * NT) {
        int ii[4], jj[4];
        S l[4], u[4], a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int x = e + q * NT;
          ii[q] = (int)(((float)x + 0.5f) * inv_m);
          jj[q] = x - ii[q] * mm;
          l[q] = Ak[ii[q] * N];
          u[q] = U[jj[q]];
          a[q] = T0[ii[q] * N + jj[q]];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) T0[ii[q] * N + jj[q]] = fma(-l[q], u[q], a[q]);
      }
      for (; e < tot; e += NT) {
        const int i = (int)(((float)e + 0.5f) * inv_m);
        const int j = e - i * mm;
        T0[i * N + j] = fma(-Ak[i * N], U[j], T0[i * N + j]);
      }
    }
    g.sync();
  }
  // compose the row interchanges: row i of the factors is row perm[i] of the original matrix
  if (g.t == 0) {
    for (int i = 0; i < N; ++i) perm[i] = i;
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  g.sync();
  return ok;
}

// x <- A^-1 x with the factors of cell_lu, by one warp with x in registers: lane l holds rows
// l, l+32, .. (S slots, N <= 32 S), so a column step is a shuffle and one FMA per slot that
// still holds rows below (forward) or above (backward) the column, without shared-memory round
// trips or barriers.  The slot loops are unrolled over compile-time bounds so that no FMA is
// issued for a slot with no active row.  perm is the composed row permutation of the LU.
// T is double (FP64 factors) or float (mixed precision; then b is scaled by 2^-er on entry and
// the result by 2^-ec on exit, see form_and_factor32).
template <int S, typename T>
__device__ void warp_lu_solve_s(const T* A, int N, const int* perm, const T* invdiag, const int* er, const int* ec,
                                const double* b, double* x) {
  const int lane = threadIdx.x & 31;
  T xr[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    T v = T(0);
    if (i < N) {
      const int pi = perm[i];
      v = er ? (T)(b[pi] * pow2(-er[pi])) : (T)b[pi];
    }
    xr[s] = v;
  }
  __syncwarp();
  // forward substitution with the unit lower factor: column j in slot jb updates slots >= jb
#pragma unroll
  for (int jb = 0; jb < S; ++jb) {
    const int jend = min(32 * jb + 32, N - 1);
    for (int j = 32 * jb; j < jend; ++j) {
      const T xj = __shfl_sync(kFull, xr[jb], j & 31);
#pragma unroll
      for (int s = jb; s < S; ++s) {
        const int i = lane + 32 * s;
        if (i > j && i < N) xr[s] = fma(-A[i * N + j], xj, xr[s]);
      }
    }
  }
  // back substitution with the upper factor: column j in slot jb updates slots <= jb
#pragma unroll
  for (int jb = S - 1; jb >= 0; --jb) {
    for (int j = min(32 * jb + 31, N - 1); j >= 32 * jb; --j) {
      const T xj = __shfl_sync(kFull, xr[jb], j & 31) * invdiag[j];
      if (lane == (j & 31)) xr[jb] = xj;
#pragma unroll
      for (int s = 0; s <= jb; ++s) {
        const int i = lane + 32 * s;
        if (i < j) xr[s] = fma(-A[i * N + j], xj, xr[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    if (i < N) x[i] = ec ? (double)xr[s] * pow2(-ec[i]) : (double)xr[s];
  }
  __syncwarp();
}

template <typename T>
__device__ void warp_lu_solve_any(const T* A, int N, const int* perm, const T* invdiag, const int* er, const int* ec,
                                  const double* b, double* x) {
  if (N <= 32) warp_lu_solve_s<1, T>(A, N, perm, invdiag, er, ec, b, x);
  else if (N <= 64) warp_lu_solve_s<2, T>(A, N, perm, invdiag, er, ec, b, x);
  else if (N <= 96) warp_lu_solve_s<3, T>(A, N, perm, invdiag, er, ec, b, x);
  else warp_lu_solve_s<4, T>(A, N, perm, invdiag, er, ec, b, x);
}

__device__ void warp_lu_solve(const double* A, int N, const int* perm, const double* invdiag, double* x) {
  warp_lu_solve_any<double>(A, N, perm, invdiag, nullptr, nullptr, x, x);
}

// Mixed precision: x <- W^-1 b through the FP32 factors of the equilibrated matrix
// S = D_r W D_c (D_r, D_c powers of two): z = D_r b, S v = z in FP32, x = D_c v.
__device__ void warp_lu_solve32(const float* A, int N, const int* perm, const float* invdiag, const int* er,
                                const int* ec, const double* b, double* x) {
  warp_lu_solve_any<float>(A, N, perm, invdiag, er, ec, b, x);
}

template <int G>
__device__ inline void cell_solve(const Grp<G>& g, const double* A, int N, const int* perm, const double* invdiag,
                                  double* x) {
  if (g.warp() == 0) warp_lu_solve(A, N, perm, invdiag, x);
  g.sync();
}

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
  int mixed;          // FP32 factors + FP64-residual refinement
  int refine_sweeps;  // refinement sweeps per stage solve (mixed)
};

// ------------------------------------------------------------------------------------------
// Mixed precision (FP32 LU + FP64-residual iterative refinement).

// Equilibrate W = I gh - J by powers of two (row exponents er, then column exponents ec, from
// the largest entries) and factor S = D_r W D_c in FP32 in the first half of buffer B.
template <int G>
__device__ bool form_and_factor32(const Grp<G>& g, const CellMem& w, int N, double gh) {
  constexpr int NT = Grp<G>::NT;
  float* S = reinterpret_cast<float*>(w.B);
  for (int i = g.t; i < N; i += NT) {
    int mx = 0;
    for (int j = 0; j < N; ++j) {
      const double v = (i == j) ? gh + w.A[i * N + j] : w.A[i * N + j];
      mx = max(mx, exp_field(v));
    }
    w.er[i] = mx - 1023;
  }
  g.sync();
  for (int j = g.t; j < N; j += NT) {
    int mx = -2100;
    for (int i = 0; i < N; ++i) {
      const double v = (i == j) ? gh + w.A[i * N + j] : w.A[i * N + j];
      const int ef = exp_field(v);
      if (ef > 0) mx = max(mx, ef - 1023 - w.er[i]);
    }
    w.ec[j] = (mx < -900) ? 0 : mx;
  }
  g.sync();
  for (int e = g.t; e < N * N; e += NT) {
    const int i = e / N, j = e - (e / N) * N;
    const double v = (i == j) ? gh + w.A[e] : w.A[e];
    S[e] = (float)(v * pow2(-w.er[i] - w.ec[j]));
  }
  g.sync();
  return cell_lu<G, float>(g, S, N, w.piv, w.perm, w.invd32);
}

// u <- W^-1 rhs.  FP64 factors: one solve.  FP32 factors: a solve, then up to refine_sweeps
// sweeps of r = rhs - W u (FP64, with the FP64 Jacobian), u += W32^-1 r, until the last
// correction is below 1e-5 of the error-control scale atol + rtol |y|.  Returns false if it
// did not get there.
template <int G>
__device__ bool stage_solve(const Grp<G>& g, const CellMem& w, const IntegrateArgs& a, int N, double gh, bool f32,
                            double* u) {
  constexpr int NT = Grp<G>::NT;
  if (!f32) {
    for (int i = g.t; i < N; i += NT) u[i] = w.rhs[i];
    g.sync();
    cell_solve(g, w.B, N, w.perm, w.invdiag, u);
    return true;
  }
  const float* S = reinterpret_cast<const float*>(w.B);
  if (g.warp() == 0) warp_lu_solve32(S, N, w.perm, w.invd32, w.er, w.ec, w.rhs, u);
  g.sync();
  double conv = INFINITY;
  for (int s = 0; s < a.refine_sweeps; ++s) {
    // residual r = rhs - W u = rhs - gh u + J u (the buffer holds -J)
    for (int i = g.t; i < N; i += NT) {
      const double* Ji = w.A + (size_t)i * N;
      double s0 = 0.0, s1 = 0.0;
      int j = 0;
      for (; j + 1 < N; j += 2) {
        s0 = fma(Ji[j], u[j], s0);
        s1 = fma(Ji[j + 1], u[j + 1], s1);
      }
      if (j < N) s0 = fma(Ji[j], u[j], s0);
      w.res[i] = fma(-gh, u[i], w.rhs[i]) - (s0 + s1);
    }
    g.sync();
    if (g.warp() == 0) warp_lu_solve32(S, N, w.perm, w.invd32, w.er, w.ec, w.res, w.res);
    g.sync();
    double c = 0.0;
    for (int i = g.t; i < N; i += NT) {
      const double d = w.res[i];
      u[i] += d;
      c = Grp<G>::nanmax(c, fabs(d) / (a.atol + a.rtol * fabs(w.y[i])));
    }
    conv = g.max_nan(c);
    if (conv <= 1e-5) break;
  }
  return conv <= 1e-5;
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
__global__ void __launch_bounds__(256, 1) integrate_kernel(DevMech m, Plan plan, IntegrateArgs a) {
  extern __shared__ double smem[];
  Grp<G> g;
  g.t = threadIdx.x % Grp<G>::NT;
  g.gid = threadIdx.x / Grp<G>::NT;
  g.parity = 0;
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
    bad = (g.sum((double)bad) > 0.0) || !(a.T[cell] > 0.0);
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
        const CellScalars s0 = cell_rates(m, g, a.p, w.y, w.f0, w, w.A, true);
        PHASE_END(0);
        cell_jacobian(m, g, s0, w.f0, w, w.A, w.B);
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
        const bool f32 = pass == 0;
        bool ok;
        if (f32) {
          ok = form_and_factor32(g, w, N, gh);
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
        conv = stage_solve(g, w, a, N, gh, f32, w.u[0]);
        PHASE_END(3);
        // stage 2
        if (conv) {
          for (int i = g.t; i < N; i += NT) w.ynew[i] = fma(c_a21, w.u[0][i], w.y[i]);
          g.sync();
          cell_rates(m, g, a.p, w.ynew, w.fs, w, nullptr, false);
          PHASE_END(4);
          for (int i = g.t; i < N; i += NT) w.rhs[i] = fma(c_c21 * invh, w.u[0][i], w.fs[i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, f32, w.u[1]);
          PHASE_END(3);
        }
        // stage 3
        if (conv) {
          for (int i = g.t; i < N; i += NT) w.ynew[i] = w.y[i] + c_a31 * w.u[0][i] + c_a32 * w.u[1][i];
          g.sync();
          cell_rates(m, g, a.p, w.ynew, w.fs, w, nullptr, false);
          PHASE_END(4);
          for (int i = g.t; i < N; i += NT)
            w.rhs[i] = w.fs[i] + invh * (c_c31 * w.u[0][i] + c_c32 * w.u[1][i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, f32, w.u[2]);
        }
        // stage 4 (same argument as stage 3)
        if (conv) {
          for (int i = g.t; i < N; i += NT)
            w.rhs[i] = w.fs[i] + invh * (c_c41 * w.u[0][i] + c_c42 * w.u[1][i] + c_c43 * w.u[2][i]);
          g.sync();
          conv = stage_solve(g, w, a, N, gh, f32, w.u[3]);
        }
        if (!conv) {
          if (g.t == 0) atomicAdd(&a.totals[3], 1ull);
          f64_until = attempt + 16;
          continue;  // redo this attempt with FP64 factors
        }
        // solution, embedded error, filtered through (I - gamma h J)^-1 = W^-1 / (gamma h)
        // (the filter only feeds the step-size control, so FP32 factors need no refinement)
        for (int i = g.t; i < N; i += NT) {
          w.ynew[i] = w.y[i] + c_m[0] * w.u[0][i] + c_m[1] * w.u[1][i] + c_m[2] * w.u[2][i] + c_m[3] * w.u[3][i];
          w.rhs[i] = c_e[0] * w.u[0][i] + c_e[1] * w.u[1][i] + c_e[2] * w.u[2][i] + c_e[3] * w.u[3][i];
        }
        g.sync();
        if (f32) {
          if (g.warp() == 0)
            warp_lu_solve32(reinterpret_cast<const float*>(w.B), N, w.perm, w.invd32, w.er, w.ec, w.rhs, w.err);
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

// One-shot source term / Jacobian for chem_rates and chem_jacobian.
template <int G>
__global__ void __launch_bounds__(256, 1) rates_kernel(DevMech m, Plan plan, double p, const double* T, const double* Y,
                                                    int64_t ncells, double* out_f, double* out_J) {
  extern __shared__ double smem[];
  Grp<G> g;
  g.t = threadIdx.x % Grp<G>::NT;
  g.gid = threadIdx.x / Grp<G>::NT;
  g.parity = 0;
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
    CellScalars s = cell_rates(m, g, p, w.y, w.f0, w, w.A, jac);
    if (jac) {
      cell_jacobian(m, g, s, w.f0, w, w.A, w.B);
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

const void* integrate_fn(int G) {
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
                Launch& L) {
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
  int max_cpc = (int)std::min<size_t>(std::max(1, std::min(8 / G, 15)), m->max_smem / per_cell);
  if (max_cpc < 1)
    return set_err(CHEM_ESIZE, "mechanism working set (" + std::to_string(per_cell) +
                                   " B per cell) exceeds the shared memory of one CTA");
  const int cpc = want_cpc > 0 ? std::min(want_cpc, max_cpc) : max_cpc;
  L.cells_per_cta = cpc;
  L.threads = 32 * G * cpc;
  L.smem = per_cell * cpc;
  const void* kernel = integ ? integrate_fn(G) : rates_fn(G);
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
    int rc = pick_launch(m, a.count, o.warps_per_cell, o.cells_per_cta, o.ctas_per_sm, true, L);
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

int chem_integrate(const chem_mech* mc, double p_Pa, double* T, double* Y, int64_t ncells, double dt, double rtol,
                   double atol, double* h_inout, int32_t* status, const chem_opts* opts, chem_stats* stats,
                   void* stream) {
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
  if (o.precision != CHEM_PREC_FP64 && o.precision != CHEM_PREC_MIXED)
    return set_err(CHEM_EINVAL, "chem_integrate: unknown precision mode");
  if (o.precision == CHEM_PREC_MIXED && (o.refine_sweeps < 1 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate: refine_sweeps must be 1..4");
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
  a.mixed = o.precision == CHEM_PREC_MIXED; a.refine_sweeps = o.refine_sweeps;
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
  if (o.precision != CHEM_PREC_FP64 && o.precision != CHEM_PREC_MIXED)
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: unknown precision mode");
  if (o.precision == CHEM_PREC_MIXED && (o.refine_sweeps < 1 || o.refine_sweeps > 4))
    return set_err(CHEM_EINVAL, "chem_integrate_noalloc: refine_sweeps must be 1..4");
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
  rc = pick_launch(m, ncells, o.warps_per_cell, o.cells_per_cta, o.ctas_per_sm, true, L);
  if (rc) return rc;
  int32_t* d_steps = reinterpret_cast<int32_t*>(s + kNoAllocCounters);
  int32_t* d_rej = d_steps + kNoAllocMaxCells;
  IntegrateArgs a;
  a.p = p_Pa * 10.0; a.dt = dt; a.rtol = rtol; a.atol = atol;
  a.T = T; a.Y = Y; a.h_inout = h_inout; a.status = status;
  a.steps_out = d_steps; a.rej_out = d_rej;
  a.totals = reinterpret_cast<unsigned long long*>(s + 64);
  a.queue = reinterpret_cast<int*>(s);
  a.ncells = ncells; a.first = 0; a.count = ncells; a.max_steps = o.max_steps; a.use_queue = o.use_queue;
  a.mixed = o.precision == CHEM_PREC_MIXED; a.refine_sweeps = o.refine_sweeps;
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
