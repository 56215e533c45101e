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
#include <string>
#include <vector>

#include "../../include/chemgpu.h"
#include "chem_internal.h"

using namespace chemgpu;

namespace {

constexpr double kRu = 8.314462618e7;  // erg/(mol K)
constexpr double kPatm = 1.01325e6;    // dyn/cm^2
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
// Per-warp shared-memory plan (doubles unless noted).

struct Plan {
  int N, K, R, n_pd;
  int SA;         // size of each of the two matrix buffers: max(N*N, 8*R)
  int off_A, off_B, off_vec, off_sp, off_q, off_M, off_piv, total;  // in doubles
};

__host__ __device__ inline int round2(int x) { return (x + 1) & ~1; }

__host__ __device__ inline Plan make_plan(int K, int R, int n_pd) {
  Plan p;
  p.N = K; p.K = K; p.R = R; p.n_pd = n_pd;
  p.SA = round2(max(K * K, 8 * R));
  p.off_A = 0;
  p.off_B = p.SA;
  p.off_vec = 2 * p.SA;
  // vectors: y, ynew, f0, fs, u0..u3, rhs, err, invdiag, zc, dwT, rowA, rowB, ccol  (16 x N)
  p.off_sp = p.off_vec + 16 * round2(K);
  // species: C, hRT, cpR, gRT, omega, dcpR  (6 x K)
  p.off_q = p.off_sp + 6 * round2(K);
  p.off_M = p.off_q + round2(R);
  p.off_piv = p.off_M + round2(max(n_pd, 1));
  p.total = p.off_piv + round2((K + 1) / 2 + 1);
  return p;
}

struct WarpMem {
  double *A, *B;
  double *y, *ynew, *f0, *fs, *u[4], *rhs, *err, *invdiag, *zc, *dwT, *rowA, *rowB, *ccol;
  double *C, *hRT, *cpR, *gRT, *omega, *dcpR;
  double *q, *M;
  int* piv;
};

__device__ inline WarpMem carve(double* base, const Plan& p) {
  WarpMem w;
  w.A = base + p.off_A;
  w.B = base + p.off_B;
  const int n = round2(p.K);
  double* v = base + p.off_vec;
  w.y = v; w.ynew = v + n; w.f0 = v + 2 * n; w.fs = v + 3 * n;
  for (int i = 0; i < 4; ++i) w.u[i] = v + (4 + i) * n;
  w.rhs = v + 8 * n; w.err = v + 9 * n; w.invdiag = v + 10 * n; w.zc = v + 11 * n; w.dwT = v + 12 * n;
  w.rowA = v + 13 * n; w.rowB = v + 14 * n; w.ccol = v + 15 * n;
  double* s = base + p.off_sp;
  w.C = s; w.hRT = s + n; w.cpR = s + 2 * n; w.gRT = s + 3 * n; w.omega = s + 4 * n; w.dcpR = s + 5 * n;
  w.q = base + p.off_q;
  w.M = base + p.off_M;
  w.piv = reinterpret_cast<int*>(base + p.off_piv);
  return w;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// max that propagates NaN (a NaN error norm must reject the step)
__device__ inline double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

__device__ inline double warp_max_nan(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// ------------------------------------------------------------------------------------------
// Thermochemistry and rates (Eq. 1).  Scalars of the cell state, identical in every lane.

struct CellScalars {
  double T, invT, lnT, rho, Wbar, cp, dcp_dT, fT, Q;
};

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
  const double e3 = exp(-T / T3), e1 = exp(-T / T1), e2 = exp(-T2 * invT);
  const double Fcent = (1.0 - a) * e3 + a * e1 + e2;
  const double L = log10(Fcent);
  const double c = -0.4 - 0.67 * L, n = 0.75 - 1.27 * L;
  const double x = log10(Pr);
  const double den = n - 0.14 * (x + c);
  const double f1 = (x + c) / den;
  const double g = 1.0 + f1 * f1;
  F = exp10(L / g);
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
__device__ CellScalars warp_rates(const DevMech& m, double p, const double* y, double* f, const WarpMem& w,
                                  double* scr, bool jac) {
  const int lane = threadIdx.x & 31;
  const int K = m.K, d = K - 1;
  CellScalars s;
  s.T = y[0];
  s.invT = 1.0 / s.T;
  s.lnT = log(s.T);
  // mass fractions, mean molar mass, density, concentrations, thermo
  double ysum = 0.0, yw = 0.0;
  for (int k = lane; k < d; k += 32) {
    const double Yk = y[1 + k];
    ysum += Yk;
    yw += Yk * m.sp[k * kSpDoubles + 1];
  }
  ysum = warp_sum(ysum);
  yw = warp_sum(yw);
  const double Yd = 1.0 - ysum;
  yw += Yd * m.sp[d * kSpDoubles + 1];
  s.Wbar = 1.0 / yw;
  s.rho = p * s.Wbar / (kRu * s.T);
  double cp = 0.0, dcp = 0.0;
  for (int k = lane; k < K; k += 32) {
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
  s.cp = warp_sum(cp) * kRu;
  s.dcp_dT = warp_sum(dcp) * kRu;
  __syncwarp();
  // third-body concentrations [M]_r = sum_k eff_rk C_k for the pressure-dependent reactions
  for (int r = lane; r < m.n_pd; r += 32) {
    const double* e = m.eff + (size_t)r * K;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += e[k] * w.C[k];
    w.M[r] = acc;
  }
  __syncwarp();
  const double ln_patm_rut = log(kPatm / (kRu * s.T));
  for (int r = lane; r < m.R; r += 32) {
    const int* ii = m.rxi + r * kRxInts;
    const double* rd = m.rxd + r * kRxDoubles;
    const int a0 = ii[0], a1 = ii[1], p0 = ii[2], p1 = ii[3];
    const double Ca0 = w.C[a0], Ca1 = (a1 >= 0) ? w.C[a1] : 1.0;
    const double Cp0 = w.C[p0], Cp1 = (p1 >= 0) ? w.C[p1] : 1.0;
    const double pf = Ca0 * Ca1, pr = Cp0 * Cp1;
    double kf = exp(rd[0] + rd[1] * s.lnT - rd[2] * s.invT);
    double dG = w.gRT[p0] - w.gRT[a0];
    if (p1 >= 0) dG += w.gRT[p1];
    if (a1 >= 0) dG -= w.gRT[a1];
    const int dnu = m.dnu[r];
    // 1/Kc = exp(sum nu g/RT - dnu ln(Patm/(Ru T)))
    const double invKc = exp(dG - dnu * ln_patm_rut);
    double mfac = 1.0, Mr = 0.0;
    double Pr = 0.0, F = 1.0, dlF = 0.0, dlnF_dT = 0.0, k0 = 0.0;
    const bool pd = r >= m.n_elem;
    const bool fo = r >= m.n_elem + m.n_tb;
    const double* fop = nullptr;
    if (pd) Mr = w.M[r - m.n_elem];
    if (fo) {
      fop = m.fo + (size_t)(r - m.n_elem - m.n_tb) * kFoDoubles;
      k0 = exp(fop[0] + fop[1] * s.lnT - fop[2] * s.invT);
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
      const double dlnkinf = rd[1] * s.invT + rd[2] * s.invT * s.invT;
      double phi = 0.0, dlnk = dlnkinf;
      if (fo) {
        const double dk_dM = k0 * F / (1.0 + Pr) * (1.0 / (1.0 + Pr) + dlF);
        phi = dk_dM * (pf - invKc * pr);
        const double dlnk0 = fop[1] * s.invT + fop[2] * s.invT * s.invT;
        dlnk = dlnkinf + (1.0 / (1.0 + Pr) + dlF) * (dlnk0 - dlnkinf) + dlnF_dT;
      } else if (pd) {
        phi = kf * pf - kr * pr;
      }
      const double dqdT = mfac * (kf * dlnk * pf - kr * (dlnk - dlnKc_dT) * pr);
      double DC = phi * Mr;
      for (int u = 0; u < 4; ++u) {
        const int j = ii[4 + u];
        double D = 0.0;
        if (j >= 0) {
          const double dpf = (a0 == j ? Ca1 : 0.0) + (a1 == j ? Ca0 : 0.0);
          const double dpr = (p0 == j ? Cp1 : 0.0) + (p1 == j ? Cp0 : 0.0);
          D = mfac * (kf * dpf - kr * dpr);
          DC += D * w.C[j];
        }
        o[u] = D;
      }
      o[4] = phi;
      o[5] = DC;
      o[6] = dqdT;
      o[7] = dH * kRu * s.T;
    }
  }
  __syncwarp();
  // species production rates and the source term
  double Qp = 0.0;
  for (int k = lane; k < K; k += 32) {
    double om = 0.0;
    for (int e = m.sr_ptr[k]; e < m.sr_ptr[k + 1]; ++e) {
      const int code = m.sr_idx[e];
      om += (double)((code & 7) - 4) * w.q[code >> 3];
    }
    w.omega[k] = om;
    Qp += w.hRT[k] * om;
    if (k < d) f[1 + k] = m.sp[k * kSpDoubles] * om / s.rho;
  }
  s.Q = warp_sum(Qp) * kRu * s.T;
  s.fT = -s.Q / (s.rho * s.cp);
  if (lane == 0) f[0] = s.fT;
  __syncwarp();
  return s;
}

// Assemble the analytical Jacobian (Sec. 2.3) at the state of the preceding warp_rates(jac)
// call.  scr (= the J buffer, overwritten) holds the per-reaction data, Z is scratch (N*N),
// J receives d f / d phi.  Chain rule through C_j = rho Y_j / W_j, rho = p Wbar/(Ru T),
// Y_K = 1 - sum Y_i; Z rows k < K-1 hold d omega_k / dC, row K-1 holds d Q / dC.
__device__ void warp_jacobian(const DevMech& m, const CellScalars& s, const double* f, const WarpMem& w, double* J,
                              double* Z) {
  const int lane = threadIdx.x & 31;
  const int K = m.K, N = K, d = K - 1;
  const double* scr = J;
  for (int e = lane; e < N * N; e += 32) Z[e] = 0.0;
  __syncwarp();
  // mass-action part: each reaction touches at most 4 rows (+ the Q row) x 4 columns
  for (int r = 0; r < m.R; ++r) {
    if (lane < 20) {
      const int* ii = m.rxi + r * kRxInts;
      const int rs = lane >> 2, cs = lane & 3;
      const int col = ii[4 + cs];
      if (col >= 0) {
        const double D = scr[(size_t)r * 8 + cs];
        if (rs < 4) {
          const int row = ii[8 + rs];
          if (row >= 0) Z[row * N + col] += (double)ii[12 + rs] * D;
        } else {
          Z[d * N + col] += scr[(size_t)r * 8 + 7] * D;
        }
      }
    }
    __syncwarp();
  }
  // efficiency part of the pressure-dependent reactions: rows x all columns
  for (int r = m.n_elem; r < m.R; ++r) {
    const int* ii = m.rxi + r * kRxInts;
    const double phi = scr[(size_t)r * 8 + 4];
    const double* e = m.eff + (size_t)(r - m.n_elem) * K;
    for (int rs = 0; rs < 5; ++rs) {
      int row;
      double coef;
      if (rs < 4) {
        row = ii[8 + rs];
        if (row < 0) continue;
        coef = (double)ii[12 + rs] * phi;
      } else {
        row = d;
        coef = scr[(size_t)r * 8 + 7] * phi;
      }
      for (int j = lane; j < K; j += 32) Z[row * N + j] += coef * e[j];
    }
    __syncwarp();
  }
  // per-species gathers of sum_j dq/dC_j C_j and dq/dT
  for (int k = lane; k < d; k += 32) {
    double zc = 0.0, dw = 0.0;
    for (int e = m.sr_ptr[k]; e < m.sr_ptr[k + 1]; ++e) {
      const int code = m.sr_idx[e];
      const double nu = (double)((code & 7) - 4);
      const int r = code >> 3;
      zc += nu * scr[(size_t)r * 8 + 5];
      dw += nu * scr[(size_t)r * 8 + 6];
    }
    w.zc[k] = zc;
    w.dwT[k] = dw;
  }
  double zqc = 0.0, dqt = 0.0;
  for (int r = lane; r < m.R; r += 32) {
    const double dh = scr[(size_t)r * 8 + 7];
    zqc += dh * scr[(size_t)r * 8 + 5];
    dqt += dh * scr[(size_t)r * 8 + 6];
  }
  zqc = warp_sum(zqc);
  dqt = warp_sum(dqt);
  double cpw = 0.0;
  for (int k = lane; k < K; k += 32) cpw += w.cpR[k] * w.omega[k];
  cpw = warp_sum(cpw) * kRu;
  __syncwarp();
  // per-row and per-column factors
  const double invWd = m.sp[d * kSpDoubles + 1];
  for (int k = lane; k < d; k += 32) {
    const double Wk = m.sp[k * kSpDoubles];
    w.rowA[k] = Wk * invWd * Z[k * N + d];
    w.rowB[k] = Wk / s.rho * (w.zc[k] - w.omega[k]);
    w.ccol[k] = -s.Wbar * (m.sp[k * kSpDoubles + 1] - invWd);
  }
  __syncwarp();
  const double rhocp = s.rho * s.cp;
  const double fT = s.fT;
  // temperature row and column, then the species block (J now overwrites the scratch)
  const double ZQd = Z[d * N + d];
  const double cpd = w.cpR[d] * invWd;
  for (int i = lane; i < d; i += 32) {
    const double ci = w.ccol[i];
    const double invWi = m.sp[i * kSpDoubles + 1];
    const double dQdY = s.rho * invWi * Z[d * N + i] - s.rho * invWd * ZQd + zqc * ci;
    const double dcpdY = (w.cpR[i] * invWi - cpd) * kRu;
    J[1 + i] = -dQdY / rhocp - fT * (ci + dcpdY / s.cp);
    const double Wk = m.sp[i * kSpDoubles];
    J[(1 + i) * N] = Wk / s.rho * (w.dwT[i] - w.zc[i] * s.invT) + f[1 + i] * s.invT;
  }
  if (lane == 0) J[0] = -(cpw + dqt - zqc * s.invT) / rhocp - fT * (-s.invT + s.dcp_dT / s.cp);
  const int nb = d * d;
  for (int e = lane; e < nb; e += 32) {
    const int k = e / d, i = e - k * d;
    const double Wk = m.sp[k * kSpDoubles];
    const double invWi = m.sp[i * kSpDoubles + 1];
    J[(1 + k) * N + 1 + i] = fma(w.rowB[k], w.ccol[i], fma(Wk * invWi, Z[k * N + i], -w.rowA[k]));
  }
  __syncwarp();
}

// ------------------------------------------------------------------------------------------
// Dense LU with partial pivoting (row interchanges, ties to the lowest row), in place, and the
// substitutions that use it (Sec. 2.3: dense LU + back substitution).  Returns false on an
// exactly zero pivot.

__device__ bool warp_lu(double* A, int N, int* piv, double* invdiag) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int k = 0; k < N; ++k) {
    // pivot: largest |a_ik|, compared as the bit patterns of |a| (monotone for non-negative)
    long long best = -1;
    int bi = N;
    for (int i = k + lane; i < N; i += 32) {
      const long long v = __double_as_longlong(fabs(A[i * N + k]));
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) piv[k] = bi;
    if (best <= 0) ok = false;  // zero (or all-zero) column: singular
    if (bi != k) {
      for (int j = lane; j < N; j += 32) {
        const double t = A[k * N + j];
        A[k * N + j] = A[bi * N + j];
        A[bi * N + j] = t;
      }
    }
    __syncwarp();
    const double inv = 1.0 / A[k * N + k];
    if (lane == 0) invdiag[k] = inv;
    for (int i = k + 1 + lane; i < N; i += 32) A[i * N + k] *= inv;
    __syncwarp();
    const int mm = N - k - 1;
    const int tot = mm * mm;
    if (tot > 0) {
      int ei = lane / mm, ej = lane - (lane / mm) * mm;
      for (int e = lane; e < tot; e += 32) {
        const int i = k + 1 + ei, j = k + 1 + ej;
        A[i * N + j] = fma(-A[i * N + k], A[k * N + j], A[i * N + j]);
        ej += 32;
        while (ej >= mm) { ej -= mm; ++ei; }
      }
    }
    __syncwarp();
  }
  return ok;
}

// x <- A^-1 x with the factors of warp_lu.
__device__ void warp_lu_solve(const double* A, int N, const int* piv, const double* invdiag, double* x) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      if (p != k) { const double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
  }
  __syncwarp();
  for (int j = 0; j < N - 1; ++j) {
    const double xj = x[j];
    for (int i = j + 1 + lane; i < N; i += 32) x[i] = fma(-A[i * N + j], xj, x[i]);
    __syncwarp();
  }
  for (int j = N - 1; j >= 0; --j) {
    const double xj = x[j] * invdiag[j];
    __syncwarp();
    if (lane == 0) x[j] = xj;
    for (int i = lane; i < j; i += 32) x[i] = fma(-A[i * N + j], xj, x[i]);
    __syncwarp();
  }
}

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
  int64_t ncells;
  int max_steps;
  int use_queue;
};

__device__ inline int64_t next_cell(const IntegrateArgs& a, int64_t& static_next, int64_t stride) {
  if (a.use_queue) {
    int c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(a.queue, 1);
    return (int64_t)__shfl_sync(kFull, c, 0);
  }
  const int64_t c = static_next;
  static_next += stride;
  return c;
}

__global__ void __launch_bounds__(256) integrate_kernel(DevMech m, Plan plan, IntegrateArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpMem w = carve(smem + (size_t)wib * plan.total, plan);
  const int N = m.N, K = m.K;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t static_next = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const double gam = c_gamma;
  for (;;) {
    const int64_t cell = next_cell(a, static_next, nwarps);
    if (cell >= a.ncells) break;
    // load the state phi = [T, Y_1..Y_{K-1}]
    bool bad = false;
    for (int i = lane; i < N; i += 32) {
      const double v = (i == 0) ? a.T[cell] : a.Y[(size_t)(i - 1) * a.ncells + cell];
      w.y[i] = v;
      bad |= !isfinite(v);
    }
    bad = __any_sync(kFull, bad) || !(a.T[cell] > 0.0);
    int status = CHEM_CELL_OK;
    int nsteps = 0, nrej = 0;
    double h_next = 0.01 * a.dt;
    if (a.h_inout) {
      const double h0 = a.h_inout[cell];
      if (h0 > 0.0) h_next = fmin(h0, a.dt);
    }
    if (bad) status = CHEM_CELL_BAD_INPUT;
    double t = 0.0, h = h_next;
    bool need_jac = true, last_rej = false;
    __syncwarp();
    for (int attempt = 0; status == CHEM_CELL_OK; ++attempt) {
      if (attempt >= a.max_steps) { status = CHEM_CELL_MAX_STEPS; break; }
      if (h_next < 1e-14 * a.dt) { status = CHEM_CELL_H_UNDERFLOW; break; }
      if (need_jac) {
        const CellScalars s0 = warp_rates(m, a.p, w.y, w.f0, w, w.A, true);
        warp_jacobian(m, s0, w.f0, w, w.A, w.B);
        need_jac = false;
      }
      // iteration matrix W = I/(gamma h) - J and its LU factors (buffer B)
      const double gh = 1.0 / (gam * h);
      for (int e = lane; e < N * N; e += 32) {
        const int i = e / N, j = e - i * N;
        w.B[e] = (i == j ? gh : 0.0) - w.A[e];
      }
      __syncwarp();
      const bool ok = warp_lu(w.B, N, w.piv, w.invdiag);
      double err = INFINITY;
      if (ok) {
        const double invh = 1.0 / h;
        // stage 1
        for (int i = lane; i < N; i += 32) w.u[0][i] = w.f0[i];
        __syncwarp();
        warp_lu_solve(w.B, N, w.piv, w.invdiag, w.u[0]);
        // stage 2
        for (int i = lane; i < N; i += 32) w.ynew[i] = w.y[i] + c_a21 * w.u[0][i];
        __syncwarp();
        warp_rates(m, a.p, w.ynew, w.fs, w, nullptr, false);
        for (int i = lane; i < N; i += 32) w.u[1][i] = w.fs[i] + (c_c21 * invh) * w.u[0][i];
        __syncwarp();
        warp_lu_solve(w.B, N, w.piv, w.invdiag, w.u[1]);
        // stage 3
        for (int i = lane; i < N; i += 32) w.ynew[i] = w.y[i] + c_a31 * w.u[0][i] + c_a32 * w.u[1][i];
        __syncwarp();
        warp_rates(m, a.p, w.ynew, w.fs, w, nullptr, false);
        for (int i = lane; i < N; i += 32)
          w.u[2][i] = w.fs[i] + invh * (c_c31 * w.u[0][i] + c_c32 * w.u[1][i]);
        __syncwarp();
        warp_lu_solve(w.B, N, w.piv, w.invdiag, w.u[2]);
        // stage 4 (same argument as stage 3)
        for (int i = lane; i < N; i += 32)
          w.u[3][i] = w.fs[i] + invh * (c_c41 * w.u[0][i] + c_c42 * w.u[1][i] + c_c43 * w.u[2][i]);
        __syncwarp();
        warp_lu_solve(w.B, N, w.piv, w.invdiag, w.u[3]);
        // solution, embedded error, filtered through (I - gamma h J)^-1 = W^-1 / (gamma h)
        for (int i = lane; i < N; i += 32) {
          w.ynew[i] = w.y[i] + c_m[0] * w.u[0][i] + c_m[1] * w.u[1][i] + c_m[2] * w.u[2][i] + c_m[3] * w.u[3][i];
          w.err[i] = c_e[0] * w.u[0][i] + c_e[1] * w.u[1][i] + c_e[2] * w.u[2][i] + c_e[3] * w.u[3][i];
        }
        __syncwarp();
        warp_lu_solve(w.B, N, w.piv, w.invdiag, w.err);
        double e = 0.0;
        for (int i = lane; i < N; i += 32) {
          const double sc = a.atol + a.rtol * fmax(fabs(w.y[i]), fabs(w.ynew[i]));
          e = nanmax(e, fabs(w.err[i] * gh) / sc);
        }
        err = warp_max_nan(e);
      }
      double fac;
      if (err <= 1.0) {
        t = (h >= a.dt - t) ? a.dt : t + h;
        for (int i = lane; i < N; i += 32) w.y[i] = w.ynew[i];
        __syncwarp();
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
    }
    // store phi and Y_K = 1 - sum
    double ysum = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double v = w.y[i];
      if (i == 0) a.T[cell] = v;
      else { a.Y[(size_t)(i - 1) * a.ncells + cell] = v; ysum += v; }
    }
    ysum = warp_sum(ysum);
    if (lane == 0) {
      if (status != CHEM_CELL_BAD_INPUT) a.Y[(size_t)(K - 1) * a.ncells + cell] = 1.0 - ysum;
      if (a.h_inout && status != CHEM_CELL_BAD_INPUT) a.h_inout[cell] = h_next;
      if (a.status) a.status[cell] = status;
      if (a.steps_out) a.steps_out[cell] = nsteps;
      if (a.rej_out) a.rej_out[cell] = nrej;
      atomicAdd(&a.totals[0], (unsigned long long)nsteps);
      atomicAdd(&a.totals[1], (unsigned long long)nrej);
      if (status != CHEM_CELL_OK) atomicAdd(&a.totals[2], 1ull);
    }
    __syncwarp();
  }
}

// One-shot source term / Jacobian for chem_rates and chem_jacobian.
__global__ void __launch_bounds__(256) rates_kernel(DevMech m, Plan plan, double p, const double* T, const double* Y,
                                                     int64_t ncells, double* out_f, double* out_J) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpMem w = carve(smem + (size_t)wib * plan.total, plan);
  const int N = m.N;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t cell = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; cell < ncells; cell += nwarps) {
    for (int i = lane; i < N; i += 32) w.y[i] = (i == 0) ? T[cell] : Y[(size_t)(i - 1) * ncells + cell];
    __syncwarp();
    const bool jac = out_J != nullptr;
    CellScalars s = warp_rates(m, p, w.y, w.f0, w, w.A, jac);
    if (jac) {
      warp_jacobian(m, s, w.f0, w, w.A, w.B);
      double* o = out_J + (size_t)cell * N * N;
      for (int e = lane; e < N * N; e += 32) o[e] = w.A[e];
    }
    if (out_f)
      for (int i = lane; i < N; i += 32) out_f[(size_t)i * ncells + cell] = w.f0[i];
    __syncwarp();
  }
}

}  // namespace

// ==========================================================================================
// Host side

struct chem_mech {
  HostMech host;
  DevMech dev;
  Plan plan;
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
  int warps_per_cta, grid;
  size_t smem;
};

int pick_launch(const chem_mech* m, int64_t ncells, int want_wpc, int want_ctas_per_sm, const void* kernel,
                Launch& L) {
  const size_t per_warp = (size_t)m->plan.total * sizeof(double);
  int max_wpc = (int)std::min<size_t>(8, m->max_smem / per_warp);
  if (max_wpc < 1)
    return set_err(CHEM_ESIZE, "mechanism working set (" + std::to_string(per_warp) +
                                   " B per cell) exceeds the shared memory of one CTA");
  int wpc = want_wpc > 0 ? std::min(want_wpc, max_wpc) : std::min(4, max_wpc);
  L.warps_per_cta = wpc;
  L.smem = per_warp * wpc;
  int occ = 0;
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32 * wpc, L.smem));
  if (occ < 1) return set_err(CHEM_ESIZE, "kernel cannot be resident with the requested shared memory");
  int cps = want_ctas_per_sm > 0 ? std::min(want_ctas_per_sm, occ) : occ;
  int64_t need = (ncells + wpc - 1) / wpc;
  L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)m->num_sms * cps));
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
  m->plan = make_plan(h.K, h.R, d.n_pd);
  if ((size_t)m->plan.total * sizeof(double) > m->max_smem) {
    chem_free_mechanism(m);
    return set_err(CHEM_ESIZE, "chem_load_mechanism: mechanism too large for one warp's shared memory");
  }
  *out = m;
  return CHEM_OK;
}

void chem_free_mechanism(chem_mech* m) {
  if (!m) return;
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
  int rc = pick_launch(m, ncells, 0, 0, (const void*)rates_kernel, L);
  if (rc) return rc;
  rates_kernel<<<L.grid, 32 * L.warps_per_cta, L.smem, st>>>(m->dev, m->plan, p_Pa * 10.0, dT, dY, ncells, df, dJ);
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
  if (o.precision != CHEM_PREC_FP64) return set_err(CHEM_EINVAL, "chem_integrate: unsupported precision mode");
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
  CK(cudaMemsetAsync(m->d_totals, 0, 4 * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(m->d_queue, 0, sizeof(int), st));
  Launch L;
  rc = pick_launch(m, ncells, o.cells_per_cta, o.ctas_per_sm, (const void*)integrate_kernel, L);
  if (rc) return rc;
  IntegrateArgs a;
  a.p = p_Pa * 10.0; a.dt = dt; a.rtol = rtol; a.atol = atol;
  a.T = dT; a.Y = dY; a.h_inout = dh; a.status = dstat;
  a.steps_out = m->d_steps; a.rej_out = m->d_rej;
  a.totals = m->d_totals; a.queue = m->d_queue;
  a.ncells = ncells; a.max_steps = o.max_steps; a.use_queue = o.use_queue;
  integrate_kernel<<<L.grid, 32 * L.warps_per_cta, L.smem, st>>>(m->dev, m->plan, a);
  CK(cudaGetLastError());
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
