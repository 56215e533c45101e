// Device building blocks of one cell's solve, shared by the forward integrator
// (chem_kernels.cu) and the discrete adjoint (adjoint.cu): cell groups, the per-cell
// shared-memory plan, thermochemistry, rates and the analytical Jacobian (Eq. 1, Sec. 2.3),
// dense LU with partial pivoting and the warp-register triangular solves.
//
// Everything here has internal linkage (an unnamed namespace), so each translation unit that
// includes it gets its own copy of the constants and tables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

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
// Dual numbers a + b e (e^2 = 0) for directional derivatives: the rate and Jacobian code is
// written once for a scalar type S and instantiated for double (the solve) and for Dual (the
// derivative of the Jacobian along a direction, needed by the discrete adjoint).  The
// constructor from double is explicit, so mixed double/Dual arithmetic goes through the
// overloads below and never through a silent conversion.

// the double versions stay visible next to the Dual overloads below
using ::fma;
using ::log;
using ::log10;

struct Dual {
  double v, d;
  Dual() = default;
  __device__ explicit Dual(double x) : v(x), d(0.0) {}
  __device__ Dual(double x, double dx) : v(x), d(dx) {}
};

template <class T>
struct is_dual : std::false_type {};
template <>
struct is_dual<Dual> : std::true_type {};

__device__ inline double val(double a) { return a; }
__device__ inline double val(const Dual& a) { return a.v; }

__device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, fma(a.v, b.d, a.d * b.v)); }
__device__ inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__device__ inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ inline Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ inline Dual operator/(double a, Dual b) {
  const double q = a / b.v;
  return Dual(q, -q * b.d / b.v);
}
__device__ inline Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
__device__ inline Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
__device__ inline Dual& operator*=(Dual& a, Dual b) { return a = a * b; }
__device__ inline Dual& operator*=(Dual& a, double b) { return a = a * b; }

// fma with at least one Dual operand: (a b + c) and its derivative a' b + a b' + c'
__device__ inline Dual fma(Dual a, Dual b, Dual c) { return Dual(fma(a.v, b.v, c.v), fma(a.v, b.d, fma(a.d, b.v, c.d))); }
__device__ inline Dual fma(double a, Dual b, Dual c) { return Dual(fma(a, b.v, c.v), fma(a, b.d, c.d)); }
__device__ inline Dual fma(Dual a, double b, Dual c) { return Dual(fma(a.v, b, c.v), fma(a.d, b, c.d)); }
__device__ inline Dual fma(Dual a, Dual b, double c) { return Dual(fma(a.v, b.v, c), fma(a.v, b.d, a.d * b.v)); }
__device__ inline Dual fma(double a, Dual b, double c) { return Dual(fma(a, b.v, c), a * b.d); }
__device__ inline Dual fma(Dual a, double b, double c) { return Dual(fma(a.v, b, c), a.d * b); }
__device__ inline Dual fma(double a, double b, Dual c) { return Dual(fma(a, b, c.v), c.d); }

__device__ inline Dual log(Dual a) { return Dual(log(a.v), a.d / a.v); }
__device__ inline Dual log10(Dual a) { return Dual(log10(a.v), a.d / (a.v * 2.302585092994045684)); }

// the S-typed constant x
template <class S>
__device__ inline S cst(double x) { return S(x); }

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
  // The single-warp work of a cell (triangular solves) runs on its lead warp and the
  // single-thread work of the LU (pivot reciprocals, the composed permutation) on its aux warp.
  // Warp w of a CTA issues on SM sub-partition w % 4, so the groups that share sub-partitions
  // take their lead warps on different ones: the FP64 pipes of all four carry the same load.
  int lead, aux;

  __device__ void init(int thread, int group) {
    t = thread;
    gid = group;
    parity = 0;
    lead = (G >= 4) ? group % G : (G == 2 ? (group >> 1) & 1 : 0);
    aux = (G > 1) ? (lead + 1) % G : 0;
  }

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
  // the same for dual numbers (value and derivative parts reduced together, same order)
  __device__ Dual sum(Dual v) const {
    sum2(v.v, v.d);
    return v;
  }
  __device__ void sum2(Dual& a, Dual& b) const {
    sum2(a.v, a.d);
    sum2(b.v, b.d);
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
  // max_nan of v, and whether any thread of the group has flag set (one exchange)
  __device__ double max_nan_any(double v, bool& flag) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
    flag = __any_sync(kFull, flag);
    if (G == 1) return v;
    double* r = red + (parity & 1) * 3 * G;
    parity++;
    if (lane() == 0) { r[2 * warp()] = v; r[2 * warp() + 1] = flag ? 1.0 : 0.0; }
    sync();
    double s = r[0];
    bool f = r[1] != 0.0;
#pragma unroll
    for (int i = 1; i < G; ++i) { s = nanmax(s, r[2 * i]); f = f || r[2 * i + 1] != 0.0; }
    flag = f;
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
  int off_A, off_B, off_vec, off_sp, off_q, off_M, off_piv, off_red, off_bc, total;
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
  p.off_bc = p.off_red + 6 * G + 2;  // reduction scratch + queue slot
  p.total = round2(p.off_bc + 10);     // broadcast slot of the cell scalars (5 values, dual-sized)
  return p;
}

struct CellMem {
  double *A, *B;
  double *y, *ynew, *f0, *fs, *u[4], *err, *invdiag, *zc, *dwT, *rowA, *rowB, *ccol, *rhs, *res;
  int *er, *ec;
  float* invd32;
  double *C, *hRT, *cpR, *gRT, *omega, *dcpR;
  double *q, *M, *red, *bc;
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
  w.bc = base + p.off_bc;
  return w;
}

// Working arrays of one rate / Jacobian evaluation (in the cell's shared memory), typed like the
// evaluation's scalars.
template <class S>
struct EvalMem {
  S *C, *hRT, *cpR, *gRT, *omega, *dcpR;  // species [K]
  S *q, *M;                               // net rates [R]; [M] of the pressure-dependent [n_pd]
  S *zc, *dwT, *rowA, *rowB, *ccol, *wq;  // Jacobian temporaries [K]
  S* pv;                                  // efficiency-pair coefficients [n_pairs]
  S* bc = nullptr;                        // broadcast slot of the cell scalars [5] (or none)
};

// The solve's evaluation arrays: the Jacobian temporaries reuse the stage vectors, which are
// free while the Jacobian is built (pv spans u0 .. res, n_pairs <= 8 round2(K)).
__device__ inline EvalMem<double> eval_mem(const CellMem& w) {
  EvalMem<double> e;
  e.C = w.C; e.hRT = w.hRT; e.cpR = w.cpR; e.gRT = w.gRT; e.omega = w.omega; e.dcpR = w.dcpR;
  e.q = w.q; e.M = w.M;
  e.zc = w.zc; e.dwT = w.dwT; e.rowA = w.rowA; e.rowB = w.rowB; e.ccol = w.ccol; e.wq = w.res;
  e.pv = w.u[0];
  e.bc = w.bc;
  return e;
}

// ------------------------------------------------------------------------------------------
// Thermochemistry and rates (Eq. 1).  Scalars of the cell state, identical in every thread.

template <class S>
struct CellScalarsT {
  S T, invT, lnT, rho, inv_rho, Wbar, cp, dcp_dT, fT;
};
using CellScalars = CellScalarsT<double>;

// 1/a by Newton's iteration for the reciprocal, r <- r + r (1 - m r), on the significand m of a
// (normalised to +-[1, 2) by replacing the exponent field): the seed is the FP32 approximate
// reciprocal (rcp.approx) of m's leading 24 bits, relative error below 2^-21; two steps in FP64
// square the error twice (below 2^-84, under the final rounding), so the result is within one
// unit in the last place of 1/a.  The exponent is then restored by an integer subtraction.  Four
// FP64 operations instead of a full division; zero, subnormal, very large, infinite and NaN
// arguments take the division.
__device__ inline double rcp_newton(double a) {
  const long long b = __double_as_longlong(a);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef < 3 || ef > 2044) return 1.0 / a;
  const long long mb = (b & (long long)0x800fffffffffffffULL) | (1023LL << 52);
  const double m = __longlong_as_double(mb);
  const unsigned hi = (unsigned)((unsigned long long)b >> 32);
  // m as a float: sign, exponent 127, the top 23 significand bits (truncated)
  const float mf = __uint_as_float((hi & 0x80000000u) | 0x3f800000u | (unsigned)((b >> 29) & 0x7fffff));
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
  // rf in +-[0.5, 1]: the same value as a double, by moving its fields
  const unsigned fb = __float_as_uint(rf);
  const long long rb = ((long long)(fb >> 31) << 63) | ((long long)(((fb >> 23) & 0xff) - 127 + 1023) << 52) |
                       ((long long)(fb & 0x7fffff) << 29);
  double r = __longlong_as_double(rb);
  double e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  e = fma(-m, r, 1.0);
  r = fma(r, e, r);
  // 1/a = r 2^-(ef - 1023); r's exponent field is 1022 or 1023, the result's stays in [1, 2043]
  return __longlong_as_double(__double_as_longlong(r) - ((long long)(ef - 1023) << 52));
}

// 1/x for the scalar types of the rate code (the fall-off quotients): Newton's reciprocal, and for
// a dual number (1/v, -d/v^2) from it.
__device__ inline double recip(double x) { return rcp_newton(x); }
__device__ inline Dual recip(Dual x) {
  const double r = rcp_newton(x.v);
  return Dual(r, -x.d * r * r);
}

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
  // |x| < 708 by an integer compare of the bit pattern with the sign masked (monotone for
  // non-negative doubles; NaN compares above), so the range check costs no FP64 instruction
  if ((__double_as_longlong(x) & 0x7fffffffffffffffLL) >= 0x4086200000000000LL) return exp(x);
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

__device__ inline Dual exp_fast(Dual x) {
  const double e = exp_fast(x.v);
  return Dual(e, e * x.d);
}

// 2^k as a double (|k| < 1000), exact.
__device__ inline double pow2(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Binary exponent of |a| (the biased exponent field; 0 for zero and subnormals).
__device__ inline int exp_field(double a) { return (int)((__double_as_longlong(a) >> 52) & 0x7ff); }

// NASA-7: cp/R, h/RT, s/R and d(cp/R)/dT.
template <class S>
__device__ inline void nasa7(const double* a, S T, S invT, S lnT, S& cpR, S& hRT, S& sR, S& dcpR) {
  cpR = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
  hRT = a[0] + T * (a[1] * 0.5 + T * (a[2] * (1.0 / 3.0) + T * (a[3] * 0.25 + T * a[4] * 0.2))) + a[5] * invT;
  sR = a[0] * lnT + T * (a[1] + T * (a[2] * 0.5 + T * (a[3] * (1.0 / 3.0) + T * a[4] * 0.25))) + a[6];
  dcpR = a[1] + T * (2.0 * a[2] + T * (3.0 * a[3] + T * 4.0 * a[4]));
}

// Troe broadening: F and d log10 F / d log10 Pr; with jac also d ln F / dT at fixed Pr.  The
// quotients share three reciprocals (of den, of g and, with jac, of Fcent ln 10, each by
// Newton's iteration) and the table carries 1/T3 and 1/T1, so nothing is divided.
template <class S>
__device__ inline void troe(const double* fo, S T, S invT, S Pr, S& F, S& dlF, S& dlnF_dT, bool jac) {
  const double a = fo[3], T2 = fo[6], iT3 = fo[8], iT1 = fo[9];
  const S e3 = exp_fast(-T * iT3), e1 = exp_fast(-T * iT1), e2 = exp_fast(-T2 * invT);
  const S Fcent = (1.0 - a) * e3 + a * e1 + e2;
  const S L = log10(Fcent);
  const S c = -0.4 - 0.67 * L, n = 0.75 - 1.27 * L;
  const S x = log10(Pr);
  const S xc = x + c;
  const S den = n - 0.14 * xc;
  const S iden = recip(den);
  const S f1 = xc * iden;
  const S g = 1.0 + f1 * f1;
  const S ig = recip(g);
  F = exp_fast(2.302585092994045684 * (L * ig));
  const S ig2 = ig * ig, iden2 = iden * iden;
  dlF = -2.0 * L * f1 * ig2 * (n * iden2);
  dlnF_dT = cst<S>(0.0);
  if (jac) {
    const S dFc = -(1.0 - a) * iT3 * e3 - a * iT1 * e1 + T2 * invT * invT * e2;
    const S dL = dFc * recip(Fcent * 2.302585092994045684);
    const S df1_dL = (-0.67 * den - xc * (-1.27 + 0.14 * 0.67)) * iden2;
    const S dlog10F_dL = ig - L * 2.0 * f1 * ig2 * df1_dL;
    dlnF_dT = 2.302585092994045684 * dlog10F_dL * dL;
  }
}

// Evaluates f(y) into f[0..N).  With jac, also leaves per-reaction derivative data in
// scr[u * R + r], u = 0..7: {dq/dC at the 4 distinct slot species, phi (coefficient of the
// efficiencies), sum_j dq/dC_j C_j, dq/dT at fixed C, reaction enthalpy (erg/mol)} (rows of R,
// so that the threads of consecutive reactions store to consecutive words), and the species
// production rates in w.omega.
// With kP (adjoint use, requires jac) it also writes P[r] = v . d f / d ln A_r for the weight
// vector v = vP (N): with q'_r = d q_r / d ln A_r (q_r for elementary and third-body
// reactions; q_r (Pr/(1+Pr) - d ln F/d ln Pr) for fall-off reactions, whose A is that of
// k_inf), P_r = (q'_r / rho) (sum_{k<K} nu_kr W_k v_Yk - v_T dH_r / cp).
template <int G, class S, bool kP = false>
__device__ CellScalarsT<S> cell_rates(const DevMech& m, const Grp<G>& g, double p, const S* y, S* f,
                                      const EvalMem<S>& w, S* scr, bool jac, const double* vP = nullptr,
                                      S* P = nullptr) {
  constexpr int NT = Grp<G>::NT;
  const int K = m.K, d = K - 1;
  CellScalarsT<S> s;
  s.T = y[0];
  // mass fractions, mean molar mass, density, concentrations, thermo
  S ysum = cst<S>(0.0), yw = cst<S>(0.0);
  for (int k = g.t; k < d; k += NT) {
    const S Yk = y[1 + k];
    ysum += Yk;
    yw += Yk * m.sp[k * kSpDoubles + 1];
  }
  g.sum2(ysum, yw);
  const S Yd = 1.0 - ysum;
  yw += Yd * m.sp[d * kSpDoubles + 1];
  // the cell scalars: ln T and three quotients.  An FP64 instruction costs a warp the same for one
  // lane as for 32, so with a broadcast slot one thread computes them for the whole group and the
  // other warps read them back instead of paying for them again (the same operations either way).
  if (G > 1 && w.bc) {
    if (g.t == 0) {
      w.bc[0] = 1.0 / s.T;
      w.bc[1] = log(s.T);
      const S Wbar = 1.0 / yw;
      w.bc[2] = Wbar;
      w.bc[3] = p * Wbar / (kRu * s.T);
      w.bc[4] = yw * kRu * s.T / p;
    }
    g.sync();
    s.invT = w.bc[0];
    s.lnT = w.bc[1];
    s.Wbar = w.bc[2];
    s.rho = w.bc[3];
    s.inv_rho = w.bc[4];
  } else {
    s.invT = 1.0 / s.T;
    s.lnT = log(s.T);
    s.Wbar = 1.0 / yw;
    s.rho = p * s.Wbar / (kRu * s.T);
    s.inv_rho = yw * kRu * s.T / p;
  }
  S cp = cst<S>(0.0), dcp = cst<S>(0.0);
  for (int k = g.t; k < K; k += NT) {
    const double* sp = m.sp + k * kSpDoubles;
    const S Yk = (k < d) ? y[1 + k] : Yd;
    w.C[k] = s.rho * Yk * sp[1];
    const double* a = (val(s.T) <= sp[2]) ? sp + 3 : sp + 10;
    S cpR, hRT, sR, dcpR;
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
    // four partial sums: independent FMA chains a quarter as long
    S a0 = cst<S>(0.0), a1 = cst<S>(0.0), a2 = cst<S>(0.0), a3 = cst<S>(0.0);
    int k = 0;
    for (; k + 3 < K; k += 4) {
      a0 = fma(e[k], w.C[k], a0);
      a1 = fma(e[k + 1], w.C[k + 1], a1);
      a2 = fma(e[k + 2], w.C[k + 2], a2);
      a3 = fma(e[k + 3], w.C[k + 3], a3);
    }
    for (; k < K; ++k) a0 = fma(e[k], w.C[k], a0);
    w.M[r] = (a0 + a1) + (a2 + a3);
  }
  g.sync();
  const S ln_patm_rut = kLnPatmRu - s.lnT;  // ln(Patm / (Ru T))
  // reactions: warp 0 takes [0, split) (the fall-off reactions, whose Troe branch is long, lead
  // the device order), the other warps [split, R); the split balances the warps' iteration costs
  // (split 0: reaction r goes to thread r mod 32 G)
#ifdef CHEM_RX_INTERLEAVED
  const int split = 0;
#else
  const int split = (G == 1) ? 0 : m.rx_split[G == 2 ? 1 : G == 4 ? 2 : 3];
#endif
  const int r_first = (split == 0) ? g.t : (g.warp() == 0) ? g.lane() : split + g.t - 32;
  const int r_end = (split == 0 || g.warp() != 0) ? m.R : split;
  const int r_step = (split == 0) ? NT : (g.warp() == 0) ? 32 : NT - 32;
  for (int r = r_first; r < r_end; r += r_step) {
    const int* ii = m.rxi + r * kRxInts;
    const double* rd = m.rxd + r * kRxDoubles;
    const int a0 = ii[0], a1 = ii[1], p0 = ii[2], p1 = ii[3];
    const S Ca0 = w.C[a0], Ca1 = (a1 >= 0) ? w.C[a1] : cst<S>(1.0);
    const S Cp0 = w.C[p0], Cp1 = (p1 >= 0) ? w.C[p1] : cst<S>(1.0);
    const S pf = Ca0 * Ca1, pr = Cp0 * Cp1;
    const S lkinf = fma(rd[1], s.lnT, rd[0]) - rd[2] * s.invT;
    S kf = exp_fast(lkinf);
    S dG = w.gRT[p0] - w.gRT[a0];
    if (p1 >= 0) dG += w.gRT[p1];
    if (a1 >= 0) dG -= w.gRT[a1];
    const int dnu = m.dnu[r];
    // 1/Kc = exp(sum nu g/RT - dnu ln(Patm/(Ru T)))
    const S invKc = exp_fast(dG - (double)dnu * ln_patm_rut);
    S mfac = cst<S>(1.0), Mr = cst<S>(0.0);
    S Pr = cst<S>(0.0), F = cst<S>(1.0), dlF = cst<S>(0.0), dlnF_dT = cst<S>(0.0), k0 = cst<S>(0.0);
    S inv1p = cst<S>(1.0);
    const bool pd = r < m.n_pd;
    const bool fo = r < m.n_fo;
    const double* fop = nullptr;
    if (pd) Mr = w.M[r];
    if (fo) {
      fop = m.fo + (size_t)r * kFoDoubles;
      // k0 / k_inf as one exponential of the difference of the logarithms (no quotient)
      const S ratio = exp_fast(fma(fop[1], s.lnT, fop[0]) - fop[2] * s.invT - lkinf);
      k0 = ratio * kf;
      Pr = ratio * Mr;
      if (fop[7] != 0.0) troe(fop, s.T, s.invT, Pr, F, dlF, dlnF_dT, jac);
      inv1p = recip(1.0 + Pr);
      kf = kf * Pr * inv1p * F;
    } else if (pd) {
      mfac = Mr;
    }
    const S kr = kf * invKc;
    const S q = mfac * (kf * pf - kr * pr);
    w.q[r] = q;
    if (jac) {
      S* o = scr + r;  // o[u * R]
      const int R = m.R;
      S dH = w.hRT[p0] - w.hRT[a0];
      if (p1 >= 0) dH += w.hRT[p1];
      if (a1 >= 0) dH -= w.hRT[a1];
      const S dlnKc_dT = (dH - (double)dnu) * s.invT;
      const S dlnkinf = (rd[1] + rd[2] * s.invT) * s.invT;
      S phi = cst<S>(0.0), dlnk = dlnkinf;
      if (fo) {
        const S dk_dM = k0 * F * inv1p * (inv1p + dlF);
        phi = dk_dM * (pf - invKc * pr);
        const S dlnk0 = (fop[1] + fop[2] * s.invT) * s.invT;
        dlnk = dlnkinf + (inv1p + dlF) * (dlnk0 - dlnkinf) + dlnF_dT;
      } else if (pd) {
        phi = kf * pf - kr * pr;
      }
      const S dqdT = mfac * (kf * dlnk * pf - kr * (dlnk - dlnKc_dT) * pr);
      S DC = phi * Mr;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = ii[4 + u];
        S D = cst<S>(0.0);
        if (j >= 0) {
          const S dpf = (a0 == j ? Ca1 : cst<S>(0.0)) + (a1 == j ? Ca0 : cst<S>(0.0));
          const S dpr = (p0 == j ? Cp1 : cst<S>(0.0)) + (p1 == j ? Cp0 : cst<S>(0.0));
          D = mfac * (kf * dpf - kr * dpr);
          DC = fma(D, w.C[j], DC);
        }
        o[u * R] = D;
      }
      o[4 * R] = phi;
      o[5 * R] = DC;
      o[6 * R] = dqdT;
      o[7 * R] = dH * kRu * s.T;
      if (kP) {
        double gw = 0.0;  // sum over the species rows of nu_kr W_k v_Yk
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = ii[8 + u];
          if (k >= 0) gw = fma(rd[3 + u] * m.sp[k * kSpDoubles], vP[1 + k], gw);
        }
        const S dq = fo ? q * (Pr * inv1p - dlF) : q;
        P[r] = dq * s.inv_rho * (gw - vP[0] * (o[7 * R] / s.cp));
      }
    }
  }
  g.sync();
  // species production rates and the source term
  S Qp = cst<S>(0.0);
  for (int k = g.t; k < K; k += NT) {
    // two partial sums (independent FMA chains) over the species' reactions
    S om0 = cst<S>(0.0), om1 = cst<S>(0.0);
    const int eb = m.sr_ptr[k], ee = m.sr_ptr[k + 1];
    int e = eb;
    for (; e + 1 < ee; e += 2) {
      om0 = fma(m.sr_nu[e], w.q[m.sr_idx[e]], om0);
      om1 = fma(m.sr_nu[e + 1], w.q[m.sr_idx[e + 1]], om1);
    }
    if (e < ee) om0 = fma(m.sr_nu[e], w.q[m.sr_idx[e]], om0);
    const S om = om0 + om1;
    w.omega[k] = om;
    Qp = fma(w.hRT[k], om, Qp);
    if (k < d) f[1 + k] = m.sp[k * kSpDoubles] * om * s.inv_rho;
  }
  const S Q = g.sum(Qp) * kRu * s.T;
  s.fT = -Q * s.inv_rho / s.cp;
  if (g.t == 0) f[0] = s.fT;
  g.sync();
  return s;
}

// Assemble the analytical Jacobian (Sec. 2.3) at the state of the preceding cell_rates(jac)
// call.  J (overwritten) holds the per-reaction data on entry, Z is N*N scratch, J receives
// -d f / d phi (stored negated, so that W = I/(gamma h) - J is a copy plus the diagonal).  Chain rule through C_j = rho Y_j / W_j, rho = p Wbar/(Ru T), Y_K = 1 - sum Y_i;
// Z rows k < K-1 hold d omega_k / dC, row K-1 holds d Q / dC (Q = sum_k H_k omega_k).
template <int G, class S>
__device__ void cell_jacobian(const DevMech& m, const Grp<G>& g, const CellScalarsT<S>& s, const S* f,
                              const EvalMem<S>& w, S* J, S* Z) {
  constexpr int NT = Grp<G>::NT;
  const int K = m.K, N = K, d = K - 1;
  const S* scr = J;
  for (int e = g.t; e < N * N; e += NT) Z[e] = cst<S>(0.0);
  g.sync();
  // mass-action part: one thread per receiving Z entry sums its contributions (a fixed plan
  // built with the mechanism; no two threads write the same entry, no atomics).  Each thread
  // takes four entries at once, NT apart, so that four independent FMA chains hide each other's
  // FP64 latency; every entry still sums its contributions in plan order.
  for (int e0 = g.t; e0 < m.zg_entries; e0 += 4 * NT) {
    int cb[4], len[4];
    S acc[4];
    int lmax = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = e0 + q * NT;
      const bool ok = e < m.zg_entries;
      cb[q] = ok ? m.zg_ptr[e] : 0;
      len[q] = ok ? m.zg_ptr[e + 1] - cb[q] : 0;
      lmax = max(lmax, len[q]);
      acc[q] = cst<S>(0.0);
    }
    for (int c = 0; c < lmax; ++c) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c < len[q]) acc[q] = fma(m.zg_coef[cb[q] + c], scr[m.zg_src[cb[q] + c]], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (e0 + q * NT < m.zg_entries) Z[m.zg_dst[e0 + q * NT]] = acc[q];
  }
  g.sync();
  // efficiency part of the pressure-dependent reactions: Z[k][j] += sum_r v_kr eff_rj over the
  // (row k, reaction r) pairs, v_kr = nu_kr phi_r.  The coefficients go to the stage-vector area
  // first (free while the Jacobian is built).
  S* v = w.pv;
  for (int c = g.t; c < m.n_pairs; c += NT) v[c] = m.pr_nu[c] * scr[4 * m.R + m.pr_pd[c]];
  g.sync();
  {
    // four (row, column) items per thread at once, NT apart (independent FMA chains); each item
    // sums its row's pairs in plan order
    const float invK = 1.0f / (float)K;
    const int items = m.n_prows * K;
    for (int x0 = g.t; x0 < items; x0 += 4 * NT) {
      int zi[4], jj[4], cb[4], len[4];
      S acc[4];
      int lmax = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int x = x0 + q * NT;
        const bool ok = x < items;
        const int ri = ok ? (int)(((float)x + 0.5f) * invK) : 0;
        jj[q] = ok ? x - ri * K : 0;
        const int row = m.pr_rows[ri];
        zi[q] = row * N + jj[q];
        cb[q] = m.pr_ptr[row];
        len[q] = ok ? m.pr_ptr[row + 1] - cb[q] : 0;
        lmax = max(lmax, len[q]);
        acc[q] = cst<S>(0.0);
      }
      for (int c = 0; c < lmax; ++c) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c < len[q]) acc[q] = fma(v[cb[q] + c], m.eff[(size_t)m.pr_pd[cb[q] + c] * K + jj[q]], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (x0 + q * NT < items) Z[zi[q]] += acc[q];
    }
  }
  g.sync();
  // per-species gathers of sum_j dq/dC_j C_j and dq/dT; enthalpy weights of the species rows
  const double invWd = m.sp[d * kSpDoubles + 1];
  const S RuT = kRu * s.T;
  S* wq = w.wq;
  for (int k = g.t; k < d; k += NT) {
    // two partial sums each (four independent FMA chains)
    S zc0 = cst<S>(0.0), dw0 = cst<S>(0.0), zc1 = cst<S>(0.0), dw1 = cst<S>(0.0);
    const int eb = m.sr_ptr[k], ee = m.sr_ptr[k + 1];
    int e = eb;
    for (; e + 1 < ee; e += 2) {
      const double nu0 = m.sr_nu[e], nu1 = m.sr_nu[e + 1];
      const int r0 = m.sr_idx[e], r1 = m.sr_idx[e + 1];
      zc0 = fma(nu0, scr[5 * m.R + r0], zc0);
      dw0 = fma(nu0, scr[6 * m.R + r0], dw0);
      zc1 = fma(nu1, scr[5 * m.R + r1], zc1);
      dw1 = fma(nu1, scr[6 * m.R + r1], dw1);
    }
    if (e < ee) {
      const double nu = m.sr_nu[e];
      const int r = m.sr_idx[e];
      zc0 = fma(nu, scr[5 * m.R + r], zc0);
      dw0 = fma(nu, scr[6 * m.R + r], dw0);
    }
    w.zc[k] = zc0 + zc1;
    w.dwT[k] = dw0 + dw1;
    // mass conservation (sum_k W_k omega_k = 0) gives omega_K = -sum_{k<K} (W_k/W_K) omega_k, so
    // Q = sum_k H_k omega_k = sum_{k<K} (H_k - H_K W_k/W_K) omega_k: the enthalpy row is a
    // weighted sum of the species rows
    wq[k] = RuT * (w.hRT[k] - w.hRT[d] * m.sp[k * kSpDoubles] * invWd);
  }
  g.sync();
  // enthalpy row Z_Q[j] = sum_k wq_k Z[k][j] (stored in row K-1), with sum_j Z_Q[j] C_j and
  // dQ/dT|_C = sum_k wq_k dw_k/dT|_C
  S zqc = cst<S>(0.0), dqt = cst<S>(0.0), cpw = cst<S>(0.0);
  for (int j = g.t; j < K; j += NT) {
    S a0 = cst<S>(0.0), a1 = cst<S>(0.0), a2 = cst<S>(0.0), a3 = cst<S>(0.0);
    int k = 0;
    for (; k + 3 < d; k += 4) {
      a0 = fma(wq[k], Z[k * N + j], a0);
      a1 = fma(wq[k + 1], Z[(k + 1) * N + j], a1);
      a2 = fma(wq[k + 2], Z[(k + 2) * N + j], a2);
      a3 = fma(wq[k + 3], Z[(k + 3) * N + j], a3);
    }
    for (; k < d; ++k) a0 = fma(wq[k], Z[k * N + j], a0);
    const S zq = (a0 + a1) + (a2 + a3);
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
  const S inv_rhocp = s.inv_rho / s.cp;
  const S inv_cp = 1.0 / s.cp;
  const S fT = s.fT;
  // temperature row and column, then the species block (J now overwrites the scratch)
  const S ZQd = Z[d * N + d];
  const S cpd = w.cpR[d] * invWd;
  for (int i = g.t; i < d; i += NT) {
    const S ci = w.ccol[i];
    const double invWi = m.sp[i * kSpDoubles + 1];
    const S dQdY = s.rho * (invWi * Z[d * N + i] - invWd * ZQd) + zqc * ci;
    const S dcpdY = (w.cpR[i] * invWi - cpd) * kRu;
    J[1 + i] = fma(dQdY, inv_rhocp, fT * (ci + dcpdY * inv_cp));
    const double Wk = m.sp[i * kSpDoubles];
    J[(1 + i) * N] = -(Wk * s.inv_rho * (w.dwT[i] - w.zc[i] * s.invT) + f[1 + i] * s.invT);
  }
  if (g.t == 0) J[0] = (cpw + dqt - zqc * s.invT) * inv_rhocp + fT * (-s.invT + s.dcp_dT * inv_cp);
  const int nb = d * d;
  const float inv_d = 1.0f / (float)d;
  // two entries per thread and iteration (independent chains), the same operations per entry
  int e = g.t;
  for (; e + NT < nb; e += 2 * NT) {
    const int k0 = (int)(((float)e + 0.5f) * inv_d), i0 = e - k0 * d;
    const int k1 = (int)(((float)(e + NT) + 0.5f) * inv_d), i1 = e + NT - k1 * d;
    const double W0 = m.sp[k0 * kSpDoubles], iW0 = m.sp[i0 * kSpDoubles + 1];
    const double W1 = m.sp[k1 * kSpDoubles], iW1 = m.sp[i1 * kSpDoubles + 1];
    const S j0 = fma(-w.rowB[k0], w.ccol[i0], fma(-W0 * iW0, Z[k0 * N + i0], w.rowA[k0]));
    const S j1 = fma(-w.rowB[k1], w.ccol[i1], fma(-W1 * iW1, Z[k1 * N + i1], w.rowA[k1]));
    J[(1 + k0) * N + 1 + i0] = j0;
    J[(1 + k1) * N + 1 + i1] = j1;
  }
  if (e < nb) {
    const int k = (int)(((float)e + 0.5f) * inv_d), i = e - k * d;
    const double Wk = m.sp[k * kSpDoubles];
    const double invWi = m.sp[i * kSpDoubles + 1];
    J[(1 + k) * N + 1 + i] = fma(-w.rowB[k], w.ccol[i], fma(-Wk * invWi, Z[k * N + i], w.rowA[k]));
  }
  g.sync();
}

// out = J^T v (J = d f / d phi at the state of the preceding cell_rates(jac) call, v a weight
// vector of length N) without forming J.  With the notation of cell_jacobian (Z = d omega/dC on
// the species rows k < K-1, a_k = W_k v_Yk, wq_k the enthalpy weights), the species block of J
// contributes -ccol_i sum_k rowB_k v_Yk - (1/W_i) t_i + (1/W_K) t_K to column i, with
// t_j = sum_k a_k Z_kj; the enthalpy row needs ZQ_j = sum_k wq_k Z_kj.  Both are weighted column
// sums of Z: per reaction, A_r = sum_rows nu_kr a_k and B_r = sum_rows nu_kr wq_k, then
// t_j = sum over the reactions with slot species j of (dq_r/dC_j) A_r + sum_pd phi_r A_r eff_rj
// (and the same with B for ZQ).  Cost O(R + contributions + n_pd K), no N x N scratch.
// ab: 2 R + 2 n_pd entries of scratch, tz: 2 K; out: N entries.
template <int G, class S>
__device__ void cell_jacobian_vjp(const DevMech& m, const Grp<G>& g, const CellScalarsT<S>& s, const S* f,
                                  const EvalMem<S>& w, const S* scr, const double* v, S* ab, S* tz, S* out) {
  constexpr int NT = Grp<G>::NT;
  const int K = m.K, R = m.R, d = K - 1, npd = m.n_pd;
  const double invWd = m.sp[d * kSpDoubles + 1];
  const S RuT = kRu * s.T;
  S* Ar = ab;
  S* Br = ab + R;
  S* fA = ab + 2 * R;
  S* fB = fA + npd;
  S* t = tz;
  S* zq = tz + K;
  // species: enthalpy weights and the gathers of sum_j dq/dC_j C_j and dq/dT
  for (int k = g.t; k < d; k += NT) {
    S zc = cst<S>(0.0), dw = cst<S>(0.0);
    for (int e = m.sr_ptr[k]; e < m.sr_ptr[k + 1]; ++e) {
      const double nu = m.sr_nu[e];
      const int r = m.sr_idx[e];
      zc = fma(nu, scr[5 * R + r], zc);
      dw = fma(nu, scr[6 * R + r], dw);
    }
    w.zc[k] = zc;
    w.dwT[k] = dw;
    w.wq[k] = RuT * (w.hRT[k] - w.hRT[d] * m.sp[k * kSpDoubles] * invWd);
  }
  g.sync();
  // per-reaction row weights
  for (int r = g.t; r < R; r += NT) {
    const int* ii = m.rxi + r * kRxInts;
    const double* rd = m.rxd + r * kRxDoubles;
    double a = 0.0;
    S b = cst<S>(0.0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = ii[8 + u];
      if (k >= 0) {
        a = fma(rd[3 + u] * m.sp[k * kSpDoubles], v[1 + k], a);
        b = fma(rd[3 + u], w.wq[k], b);
      }
    }
    Ar[r] = cst<S>(a);
    Br[r] = b;
    if (r < npd) {
      const S phi = scr[4 * R + r];
      fA[r] = phi * a;
      fB[r] = phi * b;
    }
  }
  g.sync();
  // weighted column sums t_j and ZQ_j, with sum_j ZQ_j C_j and sum_j cp_j omega_j
  S zqc = cst<S>(0.0), cpw = cst<S>(0.0);
  for (int j = g.t; j < K; j += NT) {
    S tj = cst<S>(0.0), qj = cst<S>(0.0);
    for (int e = m.cl_ptr[j]; e < m.cl_ptr[j + 1]; ++e) {
      const S D = scr[m.cl_src[e]];
      const int r = m.cl_rx[e];
      tj = fma(D, Ar[r], tj);
      qj = fma(D, Br[r], qj);
    }
    for (int p = 0; p < npd; ++p) {
      const double ej = m.eff[(size_t)p * K + j];
      tj = fma(ej, fA[p], tj);
      qj = fma(ej, fB[p], qj);
    }
    t[j] = tj;
    zq[j] = qj;
    zqc = fma(qj, w.C[j], zqc);
    cpw = fma(w.cpR[j], w.omega[j], cpw);
  }
  // species sums: sum_k a_k (zc_k - omega_k), sum_k wq_k dwT_k, and the temperature column
  S sB = cst<S>(0.0), dqt = cst<S>(0.0), sT = cst<S>(0.0);
  for (int k = g.t; k < d; k += NT) {
    const double Wk = m.sp[k * kSpDoubles];
    const double ak = Wk * v[1 + k];
    sB = fma(ak, w.zc[k] - w.omega[k], sB);
    dqt = fma(w.wq[k], w.dwT[k], dqt);
    // -J[1+k][0] (stored-negated form of cell_jacobian) times v_Yk
    const S nj = -(Wk * s.inv_rho * (w.dwT[k] - w.zc[k] * s.invT) + f[1 + k] * s.invT);
    sT = fma(nj, v[1 + k], sT);
  }
  g.sum2(zqc, cpw);
  g.sum2(sB, dqt);
  sT = g.sum(sT);
  cpw = cpw * kRu;
  sB = sB * s.inv_rho;
  g.sync();
  const S inv_rhocp = s.inv_rho / s.cp;
  const S inv_cp = 1.0 / s.cp;
  const S fT = s.fT;
  const S sA = invWd * t[d];
  const S ZQd = zq[d];
  const S cpd = w.cpR[d] * invWd;
  const double v0 = v[0];
  for (int i = g.t; i < d; i += NT) {
    const double invWi = m.sp[i * kSpDoubles + 1];
    const S ci = -s.Wbar * (invWi - invWd);
    const S dQdY = s.rho * (invWi * zq[i] - invWd * ZQd) + zqc * ci;
    const S dcpdY = (w.cpR[i] * invWi - cpd) * kRu;
    const S nj0 = fma(dQdY, inv_rhocp, fT * (ci + dcpdY * inv_cp));  // -J[0][1+i]
    const S blk = sA - ci * sB - invWi * t[i];                           // sum_k -J[1+k][1+i] v_Yk
    out[1 + i] = -fma(nj0, v0, blk);
  }
  if (g.t == 0) {
    const S nj00 = (cpw + dqt - zqc * s.invT) * inv_rhocp + fT * (-s.invT + s.dcp_dT * inv_cp);
    out[0] = -fma(nj00, v0, sT);
  }
  g.sync();
}

// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// FP32 pairs ("float-float"): a value hi + lo with |lo| <= ulp(hi) / 2 carries about 48
// significand bits in FP32 arithmetic (Dekker 1971; Knuth's two-sum and the FMA two-product),
// which GB300 issues at 64 times the FP64 rate.  The FP32 operations are the IEEE-rounded
// intrinsics, so the compiler cannot contract them and the error-free transformations stay
// exact.  Used for the factors and the substitutions of CHEM_PREC_MIXED_FF.
// Conversions between FP64 and FP32 in integer arithmetic (the FP64 pipe, which bounds the
// kernels, is not used for them).  f32_of rounds to nearest, ties to even, on the 29 bits below
// the float significand (a carry runs into the exponent); magnitudes below the smallest normal
// float give a signed zero and above the largest finite float infinity.  f64_of is exact for
// normal floats, zeros, infinities and NaNs; subnormal floats give a signed zero.
__device__ inline float f32_of(double v) {
  const long long b = __double_as_longlong(v);
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  const long long mag = b & 0x7fffffffffffffffLL;
  if (mag >= 0x7ff0000000000000LL) return __uint_as_float(sign | 0x7f800000u | (mag > 0x7ff0000000000000LL));
  const long long r = mag + 0x0fffffffLL + ((mag >> 29) & 1);
  const long long fb = (r >> 29) - ((long long)(1023 - 127) << 23);
  if (fb < (1LL << 23)) return __uint_as_float(sign);
  if (fb >= 0x7f800000LL) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | (unsigned)fb);
}
__device__ inline double f64_of(float f) {
  const unsigned fb = __float_as_uint(f);
  const unsigned e = (fb >> 23) & 0xff;
  const unsigned long long sign = (unsigned long long)(fb >> 31) << 63;
  const unsigned long long ed = (e == 0) ? 0ULL : (e == 0xff) ? 0x7ffULL : (unsigned long long)(e + 896);
  const unsigned long long mant = (e == 0) ? 0ULL : (unsigned long long)(fb & 0x7fffff) << 29;
  return __longlong_as_double((long long)(sign | (ed << 52) | mant));
}

struct FF {
  float hi, lo;
  FF() = default;
  __device__ FF(float h, float l) : hi(h), lo(l) {}
  // nearest pair to an FP64 value (hi = fl32(x), lo = fl32(x - hi); x - hi is exact in FP64).
  // This one keeps the conversion instructions: through f32_of / f64_of it put a ~300-byte stack
  // frame (local memory) on the integrate kernel.
  __device__ explicit FF(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ explicit operator double() const { return f64_of(hi) + f64_of(lo); }
};

// s + e = a + b exactly (Knuth's two-sum; no ordering of |a|, |b| needed)
__device__ inline void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// renormalise s + e (|s| >= |e|, Dekker's fast two-sum)
__device__ inline FF ff_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FF(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ inline FF operator-(FF a) { return FF(-a.hi, -a.lo); }
__device__ inline FF operator*(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);  // exact error of the leading product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_norm(p, e);
}
__device__ inline FF& operator*=(FF& a, FF b) { return a = a * b; }
// a b + c
__device__ inline FF fma(FF a, FF b, FF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  two_sum(c.hi, p, s, e);
  e = __fadd_rn(e, __fadd_rn(c.lo, pe));
  return ff_norm(s, e);
}
// a b + c for the running sums of the substitutions: the same terms as fma, without the final
// renormalisation, so the pair (s, e) has s + e = c.hi + fl(a.hi b.hi) exactly and the product's
// error and c.lo summed into e (|e| grows with the rounding errors of the sum, about the same
// error as renormalising every step; the pair is only renormalised where it is converted)
__device__ inline FF fma_acc(FF a, FF b, FF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  two_sum(c.hi, p, s, e);
  return FF(s, __fadd_rn(e, __fadd_rn(c.lo, pe)));
}
__device__ inline double fma_acc(double a, double b, double c) { return fma(a, b, c); }
__device__ inline float fma_acc(float a, float b, float c) { return fmaf(a, b, c); }
// 1 / a: the FP32 reciprocal of hi and one Newton correction r (1 - a r) in pair arithmetic
__device__ inline FF ff_recip(FF a) {
  const float r = 1.0f / a.hi;
  float e = fmaf(-a.hi, r, 1.0f);
  e = fmaf(-a.lo, r, e);
  return ff_norm(r, __fmul_rn(r, e));
}

// warp broadcast of a value held by lane l
__device__ inline double shfl(double v, int l) { return __shfl_sync(kFull, v, l); }
__device__ inline float shfl(float v, int l) { return __shfl_sync(kFull, v, l); }
__device__ inline FF shfl(FF v, int l) { return FF(__shfl_sync(kFull, v.hi, l), __shfl_sync(kFull, v.lo, l)); }

// The pivot travels through the group's argmax as a double: the value itself for FP64 and
// FP32 factors (exact), the bit pattern of the pair for FP32 pairs; lu_recip turns it into
// the reciprocal in the factor type.
__device__ inline double lu_carry(double a) { return a; }
__device__ inline double lu_carry(float a) { return f64_of(a); }
__device__ inline double lu_carry(FF a) { return __hiloint2double(__float_as_int(a.hi), __float_as_int(a.lo)); }
template <typename S>
__device__ inline S lu_recip(double c);

template <>
__device__ inline double lu_recip<double>(double c) {
#ifdef CHEM_LU_RCP_DIVISION
  return 1.0 / c;
#else
  return rcp_newton(c);
#endif
}
template <>
__device__ inline float lu_recip<float>(double c) { return 1.0f / f32_of(c); }
template <>
__device__ inline FF lu_recip<FF>(double c) {
  return ff_recip(FF(__int_as_float(__double2hiint(c)), __int_as_float(__double2loint(c))));
}

// Dense LU with partial pivoting (row interchanges, ties to the lowest row), in place, and the
// substitutions that use it (Sec. 2.3: dense LU + back substitution).  Returns false on an
// exactly zero pivot.  The factors are stored as P W = L D U': the strictly lower part holds the
// unit lower factor L, the diagonal the pivots D, invdiag their reciprocals, and the strictly
// upper part the unit upper factor U' = D^-1 U (each row of U times its pivot's reciprocal, one
// rounding, after the elimination has used it), so that neither substitution has a multiply in
// its dependent chain.

// |a| as an ordered integer key (bit pattern of a non-negative float / double)
// (the sign bit masked off in the integer pipe, so that no FP64 instruction is spent on it)
__device__ inline long long abs_key(double a) { return __double_as_longlong(a) & 0x7fffffffffffffffLL; }
__device__ inline long long abs_key(float a) { return (long long)__float_as_int(fabsf(a)); }
__device__ inline long long abs_key(FF a) { return (long long)__float_as_int(fabsf(a.hi)); }

// U' = D^-1 U: the strictly upper part of row i times invdiag[i], over the N (N - 1) / 2 entries
// in row order (each thread walks its entries in increasing order and advances its row as it goes).
template <int G, typename S>
__device__ inline void lu_unit_upper(const Grp<G>& g, S* A, int N, const S* invdiag) {
  constexpr int NT = Grp<G>::NT;
  const int tot = N * (N - 1) / 2;
  int i = 0, rs = 0;  // the row of the thread's next entry and the index of that row's first entry
  for (int e = g.t; e < tot; e += NT) {
    while (e >= rs + N - 1 - i) {
      rs += N - 1 - i;
      ++i;
    }
    A[i * N + i + 1 + e - rs] *= invdiag[i];
  }
}

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
      if (v > best) { best = v; bi = i; bv = lu_carry(a); }
    }
    g.argmax(best, bi, bv);
    // one thread (of the aux warp) takes the reciprocal of the pivot while the others swap rows
    if (g.t == 32 * g.aux) {
      piv[k] = bi;
      invdiag[k] = lu_recip<S>(bv);
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
  if (g.t == 32 * g.aux) {
    for (int i = 0; i < N; ++i) perm[i] = i;
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  lu_unit_upper(g, A, N, invdiag);
  g.sync();
  return ok;
}

// The same factorisation with two group barriers per pivot column instead of four (the same
// pivots and the same operations on every entry in the same order, so the factors are bitwise
// those of cell_lu):
//   * the pivot search of column k+1 rides on step k's trailing update: each thread that updates
//     an entry of column k+1 keeps the largest |a| it produced, the warps reduce by shuffles and
//     leave one (key, row) each in the reduction scratch, and the barrier that ends the update
//     also publishes them;
//   * every thread then combines the G candidates itself (ties to the lowest row) and takes the
//     pivot's reciprocal, so no thread waits for another to compute it;
//   * the row interchange (threads over columns) and the scaled multipliers of column k (threads
//     over rows, reading the interchanged value for the pivot row) form one phase;
//   * row k-1 of the unit upper factor is scaled during step k's update (no pass at the end).
template <int G, typename S>
__device__ bool cell_lu_fused(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag) {
  constexpr int NT = Grp<G>::NT;
  double* cand = g.red;  // [2 halves][G][3]: key bits, row and carried value of each warp's best entry
  bool ok = true;
  // pivot candidates of column 0
  {
    long long best = -1;
    int bi = N;
    double bv = 0.0;
    for (int i = g.t; i < N; i += NT) {
      const S a = A[i * N];
      const long long v = abs_key(a);
      if (v > best) { best = v; bi = i; bv = lu_carry(a); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bi, o);
      const double ov = __shfl_xor_sync(kFull, bv, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = ov; }
    }
    if (g.lane() == 0) {
      cand[3 * g.warp()] = __longlong_as_double(best);
      cand[3 * g.warp() + 1] = __int2double_rn(bi);
      cand[3 * g.warp() + 2] = bv;
    }
  }
  g.sync();
  for (int k = 0; k < N; ++k) {
    const double* cr = cand + (k & 1) * 3 * G;
    long long best = __double_as_longlong(cr[0]);
    int bi = (int)cr[1];
    double bv = cr[2];
#pragma unroll
    for (int w = 1; w < G; ++w) {
      const long long ob = __double_as_longlong(cr[3 * w]);
      const int oi = (int)cr[3 * w + 1];
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = cr[3 * w + 2]; }
    }
    if (best <= 0) ok = false;  // zero column: singular
    // interchange rows k and bi in every other column; scaled multipliers of column k (the pivot
    // row's multiplier is the old row k's entry, and the pivot moves to the diagonal)
    if (bi != k)
      for (int j = g.t; j < N; j += NT) {
        if (j == k) continue;
        const S t = A[k * N + j];
        A[k * N + j] = A[bi * N + j];
        A[bi * N + j] = t;
      }
    if (k + 1 + 32 * g.warp() < N || g.t == 0) {  // this warp scales a row, or records the pivot
      const S inv = lu_recip<S>(bv);
      if (g.t == 0) {
        piv[k] = bi;
        invdiag[k] = inv;
      }
      for (int i = k + 1 + g.t; i < N; i += NT) {
        S v;
        if (i == bi) {
          v = A[k * N + k];
          A[k * N + k] = A[bi * N + k];
        } else {
          v = A[i * N + k];
        }
        v *= inv;
        A[i * N + k] = v;
      }
    }
    g.sync();
    // row k-1 of U is final (step k-1's update was its last): U' = D^-1 U there, beside the update
    if (k > 0) {
      const S dk = invdiag[k - 1];
      for (int j = k + g.t; j < N; j += NT) A[(k - 1) * N + j] *= dk;
    }
    // trailing update: column k+1 first (its entries are the next pivot's candidates, each thread
    // keeping the largest it produced), then the other columns
    const int mm = N - k - 1;
    long long nb = -1;
    int ni = N;
    double nv = 0.0;
    if (mm > 0) {
      const S* Ak = A + (size_t)(k + 1) * N + k;  // multipliers of the trailing rows
      const S* U = A + (size_t)k * N + k + 1;     // pivot row right of the diagonal
      S* T0 = A + (size_t)(k + 1) * N + k + 1;
      const S u0 = U[0];
      for (int i = g.t; i < mm; i += NT) {
        const S r = fma(-Ak[i * N], u0, T0[i * N]);
        T0[i * N] = r;
        const long long v = abs_key(r);
        if (v > nb) { nb = v; ni = k + 1 + i; nv = lu_carry(r); }
      }
      const int mc = mm - 1;  // columns k+2 .. N-1
      const int tot = mm * mc;
      if (tot > 0) {
        const float inv_m = 1.0f / (float)mc;
        int e = g.t;
        for (; e + 3 * NT < tot; e += 4 * NT) {
          int ii[4], jj[4];
          S l[4], u[4], a[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int x = e + q * NT;
            ii[q] = (int)(((float)x + 0.5f) * inv_m);
            jj[q] = x - ii[q] * mc + 1;
            l[q] = Ak[ii[q] * N];
            u[q] = U[jj[q]];
            a[q] = T0[ii[q] * N + jj[q]];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) T0[ii[q] * N + jj[q]] = fma(-l[q], u[q], a[q]);
        }
        for (; e < tot; e += NT) {
          const int i = (int)(((float)e + 0.5f) * inv_m);
          const int j = e - i * mc + 1;
          T0[i * N + j] = fma(-Ak[i * N], U[j], T0[i * N + j]);
        }
      }
    }
    if (k + 1 < N) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(kFull, nb, o);
        const int oi = __shfl_xor_sync(kFull, ni, o);
        const double ov = __shfl_xor_sync(kFull, nv, o);
        if (ob > nb || (ob == nb && oi < ni)) { nb = ob; ni = oi; nv = ov; }
      }
      if (g.lane() == 0) {
        double* cw = cand + ((k + 1) & 1) * 3 * G;
        cw[3 * g.warp()] = __longlong_as_double(nb);
        cw[3 * g.warp() + 1] = __int2double_rn(ni);
        cw[3 * g.warp() + 2] = nv;
      }
    }
    g.sync();
  }
  // compose the row interchanges: row i of the factors is row perm[i] of the original matrix
  if (g.t == 32 * g.aux) {
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

// The same factorisation in panels of 8 columns, with the same pivots and the same operations on
// every entry in the same order (so the factors are bitwise those of cell_lu):
//   1. one warp factors the panel (rows k0.., columns k0..k0+7): pivot search by warp shuffles,
//      the row interchange inside the panel, the reciprocal, the scaled column and the rank-1
//      updates of the panel's remaining columns, with warp synchronisation only;
//   2. the group applies the panel's interchanges to every other column and, right of the panel,
//      forms U12 = L11^-1 A12 (unit lower forward substitution, one column per thread);
//   3. the group applies the panel's 8 rank-1 updates to the trailing matrix, each entry taking
//      them in pivot order.
// Three group barriers per panel instead of four per column.  perm[N] (the spare slot after the
// permutation; the plan holds K + 2 ints) carries the singular flag from the panel warp.
template <int G, typename S>
__device__ bool cell_lu_blocked(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag) {
  constexpr int NT = Grp<G>::NT;
  constexpr int NB = 8;
  int* singular = perm + N;
  const int pw = g.lead;
  for (int k0 = 0; k0 < N; k0 += NB) {
    const int k1 = min(k0 + NB, N);
    if (g.warp() == pw) {
      const int lane = g.lane();
      if (k0 == 0 && lane == 0) *singular = 0;
      for (int k = k0; k < k1; ++k) {
        long long best = -1;
        int bi = N;
        for (int i = k + lane; i < N; i += 32) {
          const long long v = abs_key(A[i * N + k]);
          if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long ob = __shfl_xor_sync(kFull, best, o);
          const int oi = __shfl_xor_sync(kFull, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi != k && lane < k1 - k0) {
          const S t = A[k * N + k0 + lane];
          A[k * N + k0 + lane] = A[bi * N + k0 + lane];
          A[bi * N + k0 + lane] = t;
        }
        __syncwarp();
        const S inv = lu_recip<S>(lu_carry(A[k * N + k]));
        if (lane == 0) {
          piv[k] = bi;
          invdiag[k] = inv;
          if (best <= 0) *singular = 1;  // zero column: singular
        }
        for (int i = k + 1 + lane; i < N; i += 32) {
          S* Ai = A + (size_t)i * N;
          S l = Ai[k];
          l *= inv;
          Ai[k] = l;
          for (int j = k + 1; j < k1; ++j) Ai[j] = fma(-l, A[k * N + j], Ai[j]);
        }
        __syncwarp();
      }
    }
    g.sync();
    for (int j = g.t; j < N; j += NT) {
      if (j >= k0 && j < k1) continue;
      for (int k = k0; k < k1; ++k) {
        const int p = piv[k];
        if (p != k) {
          const S t = A[k * N + j];
          A[k * N + j] = A[p * N + j];
          A[p * N + j] = t;
        }
      }
      if (j >= k1) {
        for (int r = k0 + 1; r < k1; ++r) {
          S acc = A[r * N + j];
          for (int c = k0; c < r; ++c) acc = fma(-A[r * N + c], A[c * N + j], acc);
          A[r * N + j] = acc;
        }
      }
    }
    g.sync();
    const int mm = N - k1;
    const int tot = mm * mm;
    if (tot > 0) {
      const float inv_m = 1.0f / (float)mm;
      const S* U = A + (size_t)k0 * N + k1;  // U12, row stride N
      // two entries per thread and iteration: independent chains of 8 updates
      int e = g.t;
      for (; e + NT < tot; e += 2 * NT) {
        const int i0 = (int)(((float)e + 0.5f) * inv_m), j0 = e - i0 * mm;
        const int i1 = (int)(((float)(e + NT) + 0.5f) * inv_m), j1 = e + NT - i1 * mm;
        S* A0 = A + (size_t)(k1 + i0) * N;
        S* A1 = A + (size_t)(k1 + i1) * N;
        S a0 = A0[k1 + j0], a1 = A1[k1 + j1];
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          if (k0 + c < k1) {
            a0 = fma(-A0[k0 + c], U[(size_t)c * N + j0], a0);
            a1 = fma(-A1[k0 + c], U[(size_t)c * N + j1], a1);
          }
        }
        A0[k1 + j0] = a0;
        A1[k1 + j1] = a1;
      }
      for (; e < tot; e += NT) {
        const int i0 = (int)(((float)e + 0.5f) * inv_m), j0 = e - i0 * mm;
        S* A0 = A + (size_t)(k1 + i0) * N;
        S a0 = A0[k1 + j0];
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (k0 + c < k1) a0 = fma(-A0[k0 + c], U[(size_t)c * N + j0], a0);
        A0[k1 + j0] = a0;
      }
    }
    g.sync();
  }
  // compose the row interchanges: row i of the factors is row perm[i] of the original matrix
  if (g.t == 32 * pw) {
    for (int i = 0; i < N; ++i) perm[i] = i;
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  lu_unit_upper(g, A, N, invdiag);
  g.sync();
  return *singular == 0;
}

// The factorisation the integrate kernels use: 0 = cell_lu (column by column), 1 = cell_lu_fused,
// 2 = cell_lu_blocked; all three give bitwise the same factors.  The default is the measured
// fastest per factor type (fused for FP64 and FP32 pairs, blocked for FP32, whose short FP32
// chains leave the barriers as the cost); CHEM_LU_VARIANT forces one for every type.
template <typename S>
__host__ __device__ constexpr int lu_variant_for() {
#ifdef CHEM_LU_VARIANT
  return CHEM_LU_VARIANT;
#else
  return std::is_same<S, float>::value ? 2 : 1;
#endif
}
template <int V, int G, typename S>
__device__ inline bool cell_lu_v(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag) {
  if constexpr (V == 1) return cell_lu_fused<G, S>(g, A, N, piv, perm, invdiag);
  else if constexpr (V == 2) return cell_lu_blocked<G, S>(g, A, N, piv, perm, invdiag);
  else return cell_lu<G, S>(g, A, N, piv, perm, invdiag);
}
// the kernels' schedule for factor type S
template <int G, typename S>
__device__ inline bool cell_lu_default(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag) {
  return cell_lu_v<lu_variant_for<S>(), G, S>(g, A, N, piv, perm, invdiag);
}
// any schedule, chosen at run time (the LU probe of the tests)
template <int G, typename S>
__device__ inline bool cell_lu_any(const Grp<G>& g, S* A, int N, int* piv, int* perm, S* invdiag, int variant) {
  if (variant == 1) return cell_lu_fused<G, S>(g, A, N, piv, perm, invdiag);
  if (variant == 2) return cell_lu_blocked<G, S>(g, A, N, piv, perm, invdiag);
  return cell_lu<G, S>(g, A, N, piv, perm, invdiag);
}

// x <- A^-1 x with the factors of cell_lu, by one warp with x in registers: lane l holds rows
// l, l+32, .. (S slots, N <= 32 S), so a column step is a shuffle and one FMA per slot that
// still holds rows below (forward) or above (backward) the column, without shared-memory round
// trips or barriers.  The slot loops are unrolled over compile-time bounds so that no FMA is
// issued for a slot with no active row.  perm is the composed row permutation of the LU.
// T is double (FP64 factors), float or FF (mixed precision; then b is scaled by 2^-er on entry
// and the result by 2^-ec on exit, the equilibration of form_and_factor_low).
// FP64 <-> the factor type of the substitutions, without FP64 conversion instructions
template <typename T>
__device__ inline T low_of(double v);
template <>
__device__ inline double low_of<double>(double v) { return v; }
template <>
__device__ inline float low_of<float>(double v) { return f32_of(v); }
template <>
__device__ inline FF low_of<FF>(double v) { return FF(v); }
__device__ inline double high_of(double v) { return v; }
__device__ inline double high_of(float v) { return f64_of(v); }
__device__ inline double high_of(FF v) { return (double)v; }

// One column step of the register substitutions of warp_lu_solve_s: broadcast x_j from its lane,
// then one FMA per slot holding a row below (forward, unit lower factor) or above (backward, unit
// upper factor) the column.
template <int S, typename T>
__device__ __forceinline__ void fwd_column(T (&xr)[S], const T* A, int N, int lane, int jb, int j) {
  const T xj = shfl(xr[jb], j & 31);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    if (s >= jb && i > j && i < N) xr[s] = fma_acc(-A[i * N + j], xj, xr[s]);
  }
}
template <int S, typename T>
__device__ __forceinline__ void bwd_column(T (&xr)[S], const T* A, int N, int lane, int jb, int j) {
  const T xj = shfl(xr[jb], j & 31);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    if (s <= jb && i < j) xr[s] = fma_acc(-A[i * N + j], xj, xr[s]);
  }
}

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
      v = er ? low_of<T>(b[pi] * pow2(-er[pi])) : low_of<T>(b[pi]);
    }
    xr[s] = v;
  }
  __syncwarp();
  // forward substitution with the unit lower factor: column j in slot jb updates slots >= jb.
  // FP32 and pair columns are unrolled four deep (their short chains leave instruction issue as
  // the cost: -11 % and -12 % solve time); FP64 columns keep the compiler's own loop (its chain is
  // the FP64 latency, and forcing an unroll factor made it 5-7 % slower)
#pragma unroll
  for (int jb = 0; jb < S; ++jb) {
    const int jend = min(32 * jb + 32, N - 1);
    if (std::is_same<T, double>::value) {
      for (int j = 32 * jb; j < jend; ++j) fwd_column<S>(xr, A, N, lane, jb, j);
    } else {
#pragma unroll 4
      for (int j = 32 * jb; j < jend; ++j) fwd_column<S>(xr, A, N, lane, jb, j);
    }
  }
  // D^-1 (all rows at once), then back substitution with the unit upper factor U': column j in
  // slot jb updates slots <= jb
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (lane + 32 * s < N) xr[s] = xr[s] * invdiag[lane + 32 * s];
#pragma unroll
  for (int jb = S - 1; jb >= 0; --jb) {
    if (std::is_same<T, double>::value) {
      for (int j = min(32 * jb + 31, N - 1); j >= 32 * jb; --j) bwd_column<S>(xr, A, N, lane, jb, j);
    } else {
#pragma unroll 4
      for (int j = min(32 * jb + 31, N - 1); j >= 32 * jb; --j) bwd_column<S>(xr, A, N, lane, jb, j);
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    if (i < N) x[i] = ec ? high_of(xr[s]) * pow2(-ec[i]) : high_of(xr[s]);
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

// x <- W^-T b with the factors of cell_lu (P W = L D U', P the row permutation perm): W^T =
// U'^T D L^T P, so U'^T v = b (forward, unit diagonal, column j of U'^T is row j of U'),
// z = D^-1 v, L^T w = z (backward, unit diagonal, column j of L^T is row j of L),
// x[perm[i]] = w[i].  One warp, x in registers as in warp_lu_solve_s; the factor rows are read
// contiguously.  b and x may alias.
template <int S>
__device__ void warp_lu_solve_t_s(const double* A, int N, const int* perm, const double* invdiag, const double* b,
                                  double* x) {
  const int lane = threadIdx.x & 31;
  double xr[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    xr[s] = (i < N) ? b[i] : 0.0;
  }
  __syncwarp();
#pragma unroll
  for (int jb = 0; jb < S; ++jb) {
    const int jend = min(32 * jb + 32, N);
    for (int j = 32 * jb; j < jend; ++j) {
      const double vj = __shfl_sync(kFull, xr[jb], j & 31);
      const double* Uj = A + (size_t)j * N;
#pragma unroll
      for (int s = jb; s < S; ++s) {
        const int i = lane + 32 * s;
        if (i > j && i < N) xr[s] = fma(-Uj[i], vj, xr[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (lane + 32 * s < N) xr[s] *= invdiag[lane + 32 * s];
#pragma unroll
  for (int jb = S - 1; jb >= 0; --jb) {
    for (int j = min(32 * jb + 31, N - 1); j >= 32 * jb; --j) {
      const double wj = __shfl_sync(kFull, xr[jb], j & 31);
      const double* Lj = A + (size_t)j * N;
#pragma unroll
      for (int s = 0; s <= jb; ++s) {
        const int i = lane + 32 * s;
        if (i < j) xr[s] = fma(-Lj[i], wj, xr[s]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = lane + 32 * s;
    if (i < N) x[perm[i]] = xr[s];
  }
  __syncwarp();
}

__device__ void warp_lu_solve_t(const double* A, int N, const int* perm, const double* invdiag, const double* b,
                                double* x) {
  if (N <= 32) warp_lu_solve_t_s<1>(A, N, perm, invdiag, b, x);
  else if (N <= 64) warp_lu_solve_t_s<2>(A, N, perm, invdiag, b, x);
  else if (N <= 96) warp_lu_solve_t_s<3>(A, N, perm, invdiag, b, x);
  else warp_lu_solve_t_s<4>(A, N, perm, invdiag, b, x);
}

template <int G>
__device__ inline void cell_solve(const Grp<G>& g, const double* A, int N, const int* perm, const double* invdiag,
                                  double* x) {
  if (g.warp() == g.lead) warp_lu_solve(A, N, perm, invdiag, x);
  g.sync();
}


}  // namespace
