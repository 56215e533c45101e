// Internal layout shared by the host table builder (mech_tables.cpp) and the kernels
// (chem_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace chemgpu {

// Reaction kinds.  Device order: Troe, Lindemann, third-body, elementary, so that lanes of one
// warp pass mostly run the same branch and the pressure-dependent reactions are 0 .. n_pd-1.
enum : int { kElementary = 0, kThirdBody = 1, kLindemann = 2, kTroe = 3 };

// Per-reaction integer record (16 ints).
//   [0..3]  slot species: reactant 0, reactant 1, product 0, product 1 (-1 = empty)
//   [4..7]  distinct slot species (the columns where dq/dC is non-zero without [M]), -1 pads
//   [8..11] rows: distinct species k < K-1 with non-zero net coefficient, -1 pads
//   [12..15] net coefficients of those rows
constexpr int kRxInts = 16;

// Per-reaction double record.
//   [0] ln A   [1] b   [2] Ea/Rc (K)   [3..6] net coefficients of the rows (as doubles)
constexpr int kRxDoubles = 7;

// Per fall-off reaction doubles: ln A0, b0, Ea0/Rc, alpha, T3, T1, T2, is_troe, 1/T3, 1/T1
constexpr int kFoDoubles = 10;

// Per species doubles: W, 1/W, Tmid, NASA low a1..a7, NASA high a1..a7
constexpr int kSpDoubles = 17;

struct HostMech {
  int K = 0, R = 0, E = 0;
  int n_elem = 0, n_tb = 0, n_fo = 0;  // counts in device order
  std::vector<int> order;              // device reaction index -> file reaction index
  std::vector<double> sp;              // [K][kSpDoubles]
  std::vector<double> rxd;             // [R][kRxDoubles]
  std::vector<int> rxi;                // [R][kRxInts]
  std::vector<int> dnu;                // [R] products minus reactants
  std::vector<double> eff;             // [n_tb + n_fo][K]
  std::vector<double> fo;              // [n_fo][kFoDoubles]
  // species -> (reaction, net coefficient) lists, all K species
  std::vector<int> sr_ptr;             // [K + 1]
  std::vector<int> sr_idx;             // reaction index (device order)
  std::vector<double> sr_nu;           // net coefficient of the species in that reaction
  // Jacobian gather plan (mass-action part).  Z entries (species row k < K-1, column j) that
  // receive contributions, each a list of (per-reaction scratch index src, coefficient):
  // Z[dst] = sum coef * s[src].  (src2 is kept for the layout and is always -1.)
  std::vector<int> zg_ptr;             // [n_entries + 1]
  std::vector<int> zg_dst;             // [n_entries] row * K + col
  std::vector<int> zg_src;             // [n_contrib]
  std::vector<int> zg_src2;            // [n_contrib]
  std::vector<double> zg_coef;         // [n_contrib]
  // Efficiency part: for each species row k < K-1, the pressure-dependent reactions in it:
  // (pd index, net coefficient)
  std::vector<int> pr_ptr;             // [K + 1]
  std::vector<int> pr_pd;
  std::vector<double> pr_nu;
  std::vector<int> pr_row;             // row of each (row, reaction) pair
  std::vector<int> pr_rows;            // rows with pairs, shortest lists first
  // Column lists (products with J^T): for species column j, the per-reaction scratch indices
  // of dq/dC_j and their reactions
  std::vector<int> cl_ptr;             // [K + 1]
  std::vector<int> cl_src;
  std::vector<int> cl_rx;
};

// Parse the mechanism text file; false + message on error.
bool parse_mechanism(const char* path, HostMech& m, std::string& err);

// Device view of the tables (all pointers into one device allocation).
struct DevMech {
  int K, R, N;
  int n_elem, n_tb, n_fo, n_pd;  // fall-off reactions are 0 .. n_fo-1, pressure-dependent 0 .. n_pd-1
  const double* sp;
  const double* rxd;
  const int* rxi;
  const int* dnu;
  const double* eff;
  const double* fo;
  const int* sr_ptr;
  const int* sr_idx;
  const double* sr_nu;
  int zg_entries;
  const int* zg_ptr;
  const int* zg_dst;
  const int* zg_src;
  const int* zg_src2;
  const double* zg_coef;
  const int* pr_ptr;
  const int* pr_pd;
  const double* pr_nu;
  const int* pr_row;
  const int* pr_rows;
  int n_pairs, n_prows;
  // reaction split of the rate evaluation for groups of 2, 4 and 8 warps (index 1, 2, 3; index 0
  // unused): warp 0 takes reactions [0, split), the other warps [split, R); 0 = interleaved
  int rx_split[4];
  const int* order;  // device reaction index -> file reaction index
  const int* cl_ptr;
  const int* cl_src;
  const int* cl_rx;
};

}  // namespace chemgpu
