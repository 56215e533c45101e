// CPU reference ("oracle") for the per-cell finite-rate chemistry solve.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-checkable statement of
// what the GPU library computes.  Only the tests, the smoke check and the benchmark's CPU
// baseline may build, load or call it; the product path never does.  It shares no code with
// the CUDA library: it has its own mechanism reader, its own constants and its own
// formulation of every step.
//
// What it computes (paper: Morev et al., "Fast reactive flow simulations using analytical
// Jacobian and dynamic load balancing in OpenFOAM", Sec. 2.1 Eq. (1) and Sec. 2.3 Eq. (2)):
//   * per cell, the constant-pressure adiabatic ideal-gas system d(phi)/dt = f(phi),
//     phi = [T, Y_1 .. Y_{K-1}], Y_K = 1 - sum of the others (Eq. 1);
//   * f from modified-Arrhenius rates, third-body and Lindemann/Troe fall-off reactions and
//     reverse rates from NASA-7 Gibbs equilibrium constants (the paper delegates these formulas
//     to pyJac, Sec. 2.3; the textbook forms used are written next to each function);
//   * the dense analytical Jacobian J = df/dphi (Sec. 2.3);
//   * integration over one flow time step with a linearly implicit method (Eq. 2) in its
//     adaptive Rosenbrock form: 4 stages, order 4 with an embedded order-3 error estimate,
//     L-stable, partial-pivot LU of (I - gamma h J) (Sec. 2.3: dense LU + back substitution).
//
// Everything is scalar FP64 loops in the order the formulas are written.  The scalar type is a
// template parameter so the same code runs with std::complex<double> (complex-step derivative
// check of the analytical Jacobian) and with an operation-counting type (the algorithmic FLOP
// count used by the benchmark's roofline).
//
// Units: cgs (mol, cm, s, erg), temperature in K, activation energies in cal/mol.
//
// Planted mistakes: compiled with -DORACLE_PLANT=n (n = 1..10) the oracle carries one
// deliberate error, marked "plant n" below, so that tests/test_oracle_planted.py can check that
// each of them fails at least one of the oracle's pins.  The default (0) is the oracle itself.

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

#include <algorithm>
#include <atomic>
#include <cctype>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

namespace oracle {

// Physical constants (CODATA 2018 gas constant; thermochemical calorie).
constexpr double kRu = 8.314462618e7;          // erg / (mol K)
constexpr double kRc = 8.314462618 / 4.184;    // cal / (mol K)
constexpr double kPatm = 1.01325e6;            // dyn / cm^2

// ----------------------------------------------------------------------------------------------
// Mechanism

struct Reaction {
  int type = 0;  // 0 elementary, 1 third body, 2 Lindemann, 3 Troe
  int reac[2] = {-1, -1};
  int prod[2] = {-1, -1};
  double A = 0, b = 0, Ea = 0;      // forward (high-pressure limit for fall-off), Ea in cal/mol
  double A0 = 0, b0 = 0, Ea0 = 0;   // low-pressure limit (fall-off)
  double troe[4] = {0, 0, 0, 0};    // alpha, T3, T1, T2
  std::vector<double> eff;          // collision efficiencies, K entries (types 1-3)
  int collider = -1;                // CHEMKIN '(+NAME)': the species that is the third body
};

struct Mech {
  int K = 0, R = 0, E = 0;
  std::vector<double> W, Tmid;
  std::vector<std::vector<int>> comp;             // [K][E]
  std::vector<std::vector<double>> alow, ahigh;   // [K][7]
  std::vector<Reaction> rx;
  // net stoichiometric coefficient nu[k][r] = (times k is a product) - (times k is a reactant)
  std::vector<std::vector<int>> nu;
};

// ----------------------------------------------------------------------------------------------
// CHEMKIN-II input (the common subset; an independent reader of the same text the library
// reads): ELEMENTS with optional /mass/, SPECIES, THERMO cards (name cols 1-18, elements
// 25-44, T ranges 46-73, coefficients in 15-column fields, high range first), REACTIONS with
// CAL/MOLE, KCAL/MOLE, JOULES/MOLE, KJOULES/MOLE or KELVINS; reversible equations, +M and (+M)
// with LOW / TROE and NAME/eff/ lists.

static std::string ck_up(std::string s) {
  std::transform(s.begin(), s.end(), s.begin(), [](unsigned char c) { return (char)std::toupper(c); });
  return s;
}

static std::string ck_strip(const std::string& s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

static double ck_num(std::string t, bool& ok) {
  for (char& c : t)
    if (c == 'd' || c == 'D') c = 'e';
  std::istringstream ss(t);
  double v = 0.0;
  ss >> v;
  ok = !ss.fail() && (ss >> std::ws).eof();
  return v;
}

static bool load_chemkin(const char* path, Mech& m, std::string& err) {
  std::ifstream in(path);
  if (!in) { err = std::string("cannot open ") + path; return false; }
  std::vector<std::string> L;
  for (std::string l; std::getline(in, l);) {
    const size_t bang = l.find('!');
    if (bang != std::string::npos) l.erase(bang);
    while (!l.empty() && (l.back() == '\r')) l.pop_back();
    L.push_back(l);
  }
  auto head = [&](const std::string& l) {
    std::istringstream ss(l);
    std::string w;
    ss >> w;
    return ck_up(w).substr(0, 4);
  };
  std::vector<std::string> elements, species;
  std::vector<double> mass;
  std::map<std::string, int> idx;
  std::vector<int> have;
  bool ok = true;
  size_t i = 0;
  // ELEMENTS, SPECIES: tokens up to END
  auto tokens_until_end = [&](std::string text) {
    std::vector<std::string> out;
    for (;;) {
      std::istringstream ss(text);
      for (std::string w; ss >> w;) {
        if (ck_up(w) == "END") return out;
        out.push_back(w);
      }
      if (++i >= L.size()) return out;
      const std::string h = head(L[i]);
      if (h == "SPEC" || h == "THER" || h == "REAC") { --i; return out; }
      text = L[i];
    }
  };
  for (; i < L.size(); ++i) {
    const std::string h = head(L[i]);
    if (h.empty()) continue;
    if (h == "ELEM") {
      std::string rest = L[i].substr(L[i].find_first_not_of(" \t"));
      rest = rest.substr(rest.find_first_of(" \t/") == std::string::npos ? rest.size() : rest.find_first_of(" \t/"));
      std::string all;
      for (const std::string& t : tokens_until_end(rest)) all += t + " ";
      // symbols, each optionally followed by /mass/
      for (size_t p = 0; p < all.size();) {
        const char c = all[p];
        if (std::isspace((unsigned char)c)) { ++p; continue; }
        if (c == '/') {
          const size_t q = all.find('/', p + 1);
          if (q == std::string::npos || elements.empty()) { err = "bad element mass"; return false; }
          mass.back() = ck_num(ck_strip(all.substr(p + 1, q - p - 1)), ok);
          if (!ok) { err = "bad element mass"; return false; }
          p = q + 1;
          continue;
        }
        size_t q = p;
        while (q < all.size() && !std::isspace((unsigned char)all[q]) && all[q] != '/') ++q;
        const std::string e = ck_up(all.substr(p, q - p));
        elements.push_back(e);
        const double m0 = e == "H" ? 1.00797 : e == "C" ? 12.01115 : e == "O" ? 15.9994 : e == "N" ? 14.0067
                        : e == "AR" ? 39.948 : e == "HE" ? 4.0026 : 0.0;
        mass.push_back(m0);
        p = q;
      }
    } else if (h == "SPEC") {
      std::string rest = L[i].substr(L[i].find_first_not_of(" \t"));
      rest = rest.substr(std::min(rest.size(), rest.find_first_of(" \t")));
      for (const std::string& t : tokens_until_end(rest)) {
        if (idx.count(ck_up(t))) { err = "duplicate species " + t; return false; }
        idx[ck_up(t)] = (int)species.size();
        species.push_back(t);
      }
    } else if (h == "THER") {
      m.K = (int)species.size();
      m.E = (int)elements.size();
      for (double x : mass)
        if (!(x > 0)) { err = "element without a mass"; return false; }
      m.W.assign(m.K, 0.0);
      m.Tmid.assign(m.K, 1000.0);
      m.comp.assign(m.K, std::vector<int>(m.E, 0));
      m.alow.assign(m.K, std::vector<double>(7));
      m.ahigh.assign(m.K, std::vector<double>(7));
      have.assign(m.K, 0);
      double tmid_default = 1000.0;
      size_t j = i + 1;
      if (j < L.size() && !(L[j].size() >= 80 && L[j][79] == '1')) {
        std::istringstream ss(L[j]);
        double a, b, c;
        if (ss >> a >> b >> c) { tmid_default = b; ++j; }
      }
      for (; j < L.size(); ++j) {
        if (head(L[j]) == "END") break;
        if (!(L[j].size() >= 80 && L[j][79] == '1')) continue;
        if (j + 3 >= L.size()) { err = "truncated thermo card"; return false; }
        std::istringstream ns(L[j].substr(0, 18));
        std::string name;
        ns >> name;
        auto it = idx.find(ck_up(name));
        if (it == idx.end()) { j += 3; continue; }
        const int k = it->second;
        for (int e = 0; e < 4; ++e) {
          const std::string sym = ck_up(ck_strip(L[j].substr(24 + 5 * e, 2)));
          if (sym.empty()) continue;
          const double n = ck_num(ck_strip(L[j].substr(26 + 5 * e, 3)), ok);
          if (!ok) { err = "bad element count for " + name; return false; }
          const auto pos = std::find(elements.begin(), elements.end(), sym);
          if (pos == elements.end()) {
            if (n != 0) { err = "undeclared element " + sym; return false; }
            continue;
          }
          m.comp[k][pos - elements.begin()] += (int)std::lround(n);
        }
        const std::string tm = L[j].size() >= 73 ? ck_strip(L[j].substr(65, 8)) : std::string();
        m.Tmid[k] = tm.empty() ? tmid_default : ck_num(tm, ok);
        if (!ok) { err = "bad Tmid for " + name; return false; }
        std::vector<double> a;
        for (int r = 1; r <= 3; ++r)
          for (int f = 0; f < 5 && (int)a.size() < 14; ++f) {
            if ((int)L[j + r].size() < 15 * (f + 1)) { err = "short thermo card for " + name; return false; }
            a.push_back(ck_num(ck_strip(L[j + r].substr(15 * f, 15)), ok));
            if (!ok) { err = "bad thermo coefficient for " + name; return false; }
          }
        for (int q = 0; q < 7; ++q) { m.ahigh[k][q] = a[q]; m.alow[k][q] = a[7 + q]; }
        have[k] = 1;
        j += 3;
      }
      for (int k = 0; k < m.K; ++k) {
        if (!have[k]) { err = "no thermo data for " + species[k]; return false; }
        for (int e = 0; e < m.E; ++e) m.W[k] += m.comp[k][e] * mass[e];
      }
      i = j;
    } else if (h == "REAC") {
      double to_cal = 1.0;
      {
        std::istringstream ss(L[i]);
        std::string w;
        ss >> w;
        while (ss >> w) {
          const std::string u = ck_up(w);
          if (u == "KCAL/MOLE") to_cal = 1000.0;
          else if (u == "JOULES/MOLE") to_cal = 1.0 / 4.184;
          else if (u == "KJOULES/MOLE") to_cal = 1000.0 / 4.184;
          else if (u == "KELVINS") to_cal = kRc;
          else if (u != "CAL/MOLE" && u != "MOLES") { err = "unsupported unit " + w; return false; }
        }
      }
      for (++i; i < L.size(); ++i) {
        const std::string l = ck_strip(L[i]);
        if (l.empty()) continue;
        if (head(l) == "END") break;
        if (l.find('=') != std::string::npos) {
          std::istringstream ss(l);
          std::vector<std::string> t;
          for (std::string w; ss >> w;) t.push_back(w);
          if (t.size() < 4) { err = "bad reaction: " + l; return false; }
          Reaction x;
          bool o1, o2, o3;
          x.A = ck_num(t[t.size() - 3], o1);
          x.b = ck_num(t[t.size() - 2], o2);
          x.Ea = ck_num(t[t.size() - 1], o3) * to_cal;
          if (!(o1 && o2 && o3)) { err = "bad Arrhenius parameters: " + l; return false; }
          std::string eq;
          for (size_t q = 0; q + 3 < t.size(); ++q) eq += ck_up(t[q]);
          std::string lhs, rhs;
          if (eq.find("<=>") != std::string::npos) {
            lhs = eq.substr(0, eq.find("<=>"));
            rhs = eq.substr(eq.find("<=>") + 3);
          } else if (eq.find("=>") != std::string::npos) {
            err = "irreversible reactions are not supported: " + eq;
            return false;
          } else {
            lhs = eq.substr(0, eq.find('='));
            rhs = eq.substr(eq.find('=') + 1);
          }
          int kind[2] = {0, 0};  // 1: +M, 2: (+M) or (+NAME)
          int named[2] = {-1, -1};
          std::vector<int> mols[2];
          std::string sides[2] = {lhs, rhs};
          for (int sd = 0; sd < 2; ++sd) {
            std::string sv = sides[sd];
            const size_t open = sv.find("(+");
            if (open != std::string::npos) {
              // fall-off: '(+M)' at the end of the side, or '(+NAME)' for one species as the
              // third body (CHEMKIN convention: efficiency 1 for it, 0 for every other species)
              if (sv.back() != ')') { err = "bad third body in " + eq; return false; }
              const std::string who = sv.substr(open + 2, sv.size() - open - 3);
              if (who != "M") {
                auto it = idx.find(who);
                if (it == idx.end()) { err = "unknown third body " + who; return false; }
                named[sd] = it->second;
              }
              kind[sd] = 2;
              sv.erase(open);
            }
            std::stringstream ts(sv);
            for (std::string term; std::getline(ts, term, '+');) {
              if (term.empty()) { err = "empty term in " + eq; return false; }
              if (term == "M") { kind[sd] = 1; continue; }
              int coef = 1;
              size_t d = 0;
              while (d < term.size() && std::isdigit((unsigned char)term[d])) ++d;
              if (d) coef = std::stoi(term.substr(0, d));
              auto it = idx.find(term.substr(d));
              if (it == idx.end()) { err = "unknown species " + term.substr(d); return false; }
              while (coef-- > 0) mols[sd].push_back(it->second);
            }
          }
          if (kind[0] != kind[1] || named[0] != named[1]) { err = "unbalanced third body in " + eq; return false; }
          for (int sd = 0; sd < 2; ++sd)
            if (mols[sd].empty() || mols[sd].size() > 2) { err = "one or two molecules per side: " + eq; return false; }
          x.reac[0] = mols[0][0]; x.reac[1] = mols[0].size() == 2 ? mols[0][1] : -1;
          x.prod[0] = mols[1][0]; x.prod[1] = mols[1].size() == 2 ? mols[1][1] : -1;
          x.type = kind[0] == 2 ? 2 : kind[0];
          x.collider = named[0];
          if (x.type >= 1) {
            x.eff.assign(m.K, x.collider >= 0 ? 0.0 : 1.0);
            if (x.collider >= 0) x.eff[x.collider] = 1.0;
          }
          m.rx.push_back(x);
          continue;
        }
        if (m.rx.empty()) { err = "auxiliary line before a reaction: " + l; return false; }
        Reaction& x = m.rx.back();
        const std::string ul = ck_up(l);
        std::string key = ul.substr(0, ul.find_first_of(" /"));
        auto between_slashes = [&]() {
          std::vector<double> v;
          const size_t a = l.find('/'), b = l.rfind('/');
          if (a == std::string::npos || b <= a) return v;
          std::istringstream ss(l.substr(a + 1, b - a - 1));
          for (std::string w; ss >> w;) {
            bool okw;
            v.push_back(ck_num(w, okw));
            if (!okw) return std::vector<double>();
          }
          return v;
        };
        if (key == "DUP" || key == "DUPLICATE") continue;
        if (key == "LOW") {
          const std::vector<double> v = between_slashes();
          if (x.type < 2 || v.size() != 3) { err = "bad LOW: " + l; return false; }
          x.A0 = v[0]; x.b0 = v[1]; x.Ea0 = v[2] * to_cal;
        } else if (key == "TROE") {
          const std::vector<double> v = between_slashes();
          if (x.type < 2 || (v.size() != 3 && v.size() != 4)) { err = "bad TROE: " + l; return false; }
          x.type = 3;
          x.troe[0] = v[0]; x.troe[1] = v[1]; x.troe[2] = v[2];
          x.troe[3] = v.size() == 4 ? v[3] : 1e30;
        } else if (key == "REV" || key == "PLOG" || key == "SRI" || key == "HIGH" || key == "FORD" ||
                   key == "RORD" || key == "CHEB") {
          err = "unsupported keyword " + key;
          return false;
        } else {
          if (x.type < 1) { err = "efficiencies without a third body: " + l; return false; }
          if (x.collider >= 0) { err = "efficiencies with a named third body: " + l; return false; }
          // NAME/value/ pairs
          std::string rest = l;
          while (!ck_strip(rest).empty()) {
            const size_t a = rest.find('/');
            const size_t b = rest.find('/', a + 1);
            if (a == std::string::npos || b == std::string::npos) { err = "bad efficiencies: " + l; return false; }
            auto it = idx.find(ck_up(ck_strip(rest.substr(0, a))));
            if (it == idx.end()) { err = "unknown species in efficiencies: " + l; return false; }
            x.eff[it->second] = ck_num(ck_strip(rest.substr(a + 1, b - a - 1)), ok);
            if (!ok) { err = "bad efficiency value: " + l; return false; }
            rest = rest.substr(b + 1);
          }
        }
      }
    }
  }
  if (m.K < 2 || m.rx.empty()) { err = "need SPECIES, THERMO and REACTIONS"; return false; }
  for (const Reaction& x : m.rx)
    if (x.type >= 2 && !(x.A0 > 0)) { err = "fall-off reaction without LOW"; return false; }
  m.R = (int)m.rx.size();
  m.nu.assign(m.K, std::vector<int>(m.R, 0));
  for (int r = 0; r < m.R; ++r)
    for (int s = 0; s < 2; ++s) {
      if (m.rx[r].reac[s] >= 0) m.nu[m.rx[r].reac[s]][r] -= 1;
      if (m.rx[r].prod[s] >= 0) m.nu[m.rx[r].prod[s]][r] += 1;
    }
  return true;
}

static bool load_mech(const char* path, Mech& m, std::string& err) {
  {
    std::ifstream probe(path);
    for (std::string l; std::getline(probe, l);) {
      const std::string t = ck_strip(l);
      if (t.empty() || t[0] == '#' || t[0] == '!') continue;
      if (t.rfind("CHEMMECH", 0) != 0) return load_chemkin(path, m, err);
      break;
    }
  }
  std::ifstream in(path);
  if (!in) { err = std::string("cannot open ") + path; return false; }
  std::vector<std::string> lines;
  std::string line;
  while (std::getline(in, line)) {
    size_t p = line.find_first_not_of(" \t\r");
    if (p == std::string::npos || line[p] == '#') continue;
    lines.push_back(line);
  }
  size_t li = 0;
  auto next = [&](std::istringstream& ss) -> bool {
    if (li >= lines.size()) return false;
    ss.clear();
    ss.str(lines[li++]);
    return true;
  };
  std::istringstream ss;
  std::string tok;
  if (!next(ss) || !(ss >> tok) || tok != "CHEMMECH") { err = "missing CHEMMECH header"; return false; }
  if (!next(ss) || !(ss >> tok >> m.E) || tok != "elements") { err = "bad elements line"; return false; }
  for (int e = 0; e < m.E; ++e) next(ss);
  if (!next(ss) || !(ss >> tok >> m.K) || tok != "species" || m.K < 2) { err = "bad species line"; return false; }
  m.W.resize(m.K); m.Tmid.resize(m.K);
  m.comp.assign(m.K, std::vector<int>(m.E));
  m.alow.assign(m.K, std::vector<double>(7));
  m.ahigh.assign(m.K, std::vector<double>(7));
  for (int k = 0; k < m.K; ++k) {
    double tlo, thi;
    if (!next(ss) || !(ss >> tok >> m.W[k] >> tlo >> m.Tmid[k] >> thi)) { err = "bad species record"; return false; }
    for (int e = 0; e < m.E; ++e) ss >> m.comp[k][e];
    for (int i = 0; i < 7; ++i) ss >> m.alow[k][i];
    for (int i = 0; i < 7; ++i) ss >> m.ahigh[k][i];
    if (!ss) { err = "short species record"; return false; }
  }
  if (!next(ss) || !(ss >> tok >> m.R) || tok != "reactions" || m.R < 0) { err = "bad reactions line"; return false; }
  m.rx.resize(m.R);
  for (int r = 0; r < m.R; ++r) {
    Reaction& x = m.rx[r];
    int nr, np;
    if (!next(ss) || !(ss >> x.type >> nr >> x.reac[0] >> x.reac[1] >> np >> x.prod[0] >> x.prod[1] >> x.A >> x.b >> x.Ea)) {
      err = "bad reaction record"; return false;
    }
    if (x.type >= 1) {
      if (!next(ss) || !(ss >> tok) || tok != "eff") { err = "missing eff"; return false; }
      x.eff.resize(m.K);
      for (int k = 0; k < m.K; ++k) ss >> x.eff[k];
    }
    if (x.type >= 2) {
      if (!next(ss) || !(ss >> tok >> x.A0 >> x.b0 >> x.Ea0) || tok != "low") { err = "missing low"; return false; }
    }
    if (x.type == 3) {
      if (!next(ss) || !(ss >> tok >> x.troe[0] >> x.troe[1] >> x.troe[2] >> x.troe[3]) || tok != "troe") {
        err = "missing troe"; return false;
      }
    }
  }
  m.nu.assign(m.K, std::vector<int>(m.R, 0));
  for (int r = 0; r < m.R; ++r) {
    for (int s = 0; s < 2; ++s) {
      if (m.rx[r].reac[s] >= 0) m.nu[m.rx[r].reac[s]][r] -= 1;
      if (m.rx[r].prod[s] >= 0) m.nu[m.rx[r].prod[s]][r] += 1;
    }
  }
  return true;
}

// ----------------------------------------------------------------------------------------------
// Scalar helpers: the same source runs with double, complex<double> and an op-counting type.

inline double re(double x) { return x; }
inline double re(const std::complex<double>& x) { return x.real(); }

struct OpCounts {
  int64_t add = 0, mul = 0, div = 0, exp = 0, log = 0;
};
static thread_local OpCounts g_ops;

// A double that tallies each arithmetic operation and elementary function call.
struct Cnt {
  double v;
  Cnt(double x = 0.0) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt& operator*=(Cnt& a, Cnt b) { a = a * b; return a; }
inline Cnt& operator/=(Cnt& a, Cnt b) { a = a / b; return a; }
inline Cnt exp(Cnt a) { g_ops.exp++; return Cnt(std::exp(a.v)); }
inline Cnt log(Cnt a) { g_ops.log++; return Cnt(std::log(a.v)); }
inline double re(const Cnt& x) { return x.v; }

// Forward-mode dual number (value, derivative along one direction) for the tangent-linear
// (forward sensitivity) runs.
struct Dual {
  double v, d;
  Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual& operator/=(Dual& a, Dual b) { a = a / b; return a; }
inline Dual exp(Dual a) { const double e = std::exp(a.v); return Dual(e, a.d * e); }
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline double re(const Dual& x) { return x.v; }

using std::exp;
using std::log;

template <class S>
inline S log10_(const S& x) { return log(x) / S(std::log(10.0)); }
template <class S>
inline S pow10_(const S& x) { return exp(x * S(std::log(10.0))); }

// ----------------------------------------------------------------------------------------------
// Thermodynamics: NASA 7-coefficient polynomials (McBride, Gordon & Reno, NASA TM-4513):
//   cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
//   h/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
//   s/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
// low coefficients for T <= Tmid, high above; no clamping outside the fitted range.

template <class S>
struct Thermo {
  std::vector<S> cp_R, h_RT, s_R, dcp_RdT;
};

template <class S>
static void thermo(const Mech& m, const S& T, Thermo<S>& th) {
  th.cp_R.resize(m.K); th.h_RT.resize(m.K); th.s_R.resize(m.K); th.dcp_RdT.resize(m.K);
  S lnT = log(T);
  for (int k = 0; k < m.K; ++k) {
    const std::vector<double>& a = (re(T) <= m.Tmid[k]) ? m.alow[k] : m.ahigh[k];
    th.cp_R[k] = S(a[0]) + S(a[1]) * T + S(a[2]) * T * T + S(a[3]) * T * T * T + S(a[4]) * T * T * T * T;
    th.h_RT[k] = S(a[0]) + S(a[1]) * T / S(2.0) + S(a[2]) * T * T / S(ORACLE_PLANT == 4 ? 2.0 : 3.0) +
                 S(a[3]) * T * T * T / S(4.0) + S(a[4]) * T * T * T * T / S(5.0) + S(a[5]) / T;  // plant 4
    th.s_R[k] = S(a[0]) * lnT + S(a[1]) * T + S(a[2]) * T * T / S(2.0) + S(a[3]) * T * T * T / S(3.0) +
                S(a[4]) * T * T * T * T / S(4.0) + S(a[6]);
    th.dcp_RdT[k] = S(a[1]) + S(2.0) * S(a[2]) * T + S(3.0) * S(a[3]) * T * T + S(4.0) * S(a[4]) * T * T * T;
  }
}

// ----------------------------------------------------------------------------------------------
// Rates and the source term f (Eq. 1).
//
//   k_f = A T^b exp(-Ea / (Rc T))                                         (modified Arrhenius)
//   [M] = sum_k eff_k C_k                                                  (third body)
//   fall-off (Lindemann; Troe form of Gilbert, Luther & Troe 1983, as in the CHEMKIN manual):
//     Pr = k0 [M] / kinf,   k = kinf Pr/(1+Pr) F
//     Lindemann F = 1; Troe: Fcent = (1-a) exp(-T/T3) + a exp(-T/T1) + exp(-T2/T),
//       c = -0.4 - 0.67 log10 Fcent, n = 0.75 - 1.27 log10 Fcent,
//       f1 = (log10 Pr + c) / (n - 0.14 (log10 Pr + c)),  log10 F = log10 Fcent / (1 + f1^2)
//   Kc = exp(-sum_k nu_k g_k/RT) (Patm / (Ru T))^(sum_k nu_k),   k_r = k_f / Kc
//   q = k_f prod C_reac - k_r prod C_prod   (times [M] for third-body reactions)
//   omega_k = sum_r nu_kr q_r
//   dT/dt = -sum_k H_k omega_k / (rho cp),  dY_k/dt = W_k omega_k / rho   (k < K)

template <class S>
struct RateState {
  S T, rho, Wbar, cp_mass;
  std::vector<S> Y, C;               // all K species
  Thermo<S> th;
  std::vector<S> kf, kr, M, qf, qr, q, omega;
  // fall-off helpers
  std::vector<S> Pr, F, dlogF_dlogPr, k0, kinf;
};

template <class S>
static void troe_F(const Reaction& x, const S& T, const S& Pr, S& F, S& dlog10F_dlog10Pr) {
  if (x.type == 2) { F = S(1.0); dlog10F_dlog10Pr = S(0.0); return; }
  const double a = x.troe[0], T3 = x.troe[1], T1 = x.troe[2], T2 = x.troe[3];
  S Fcent = S(1.0 - a) * exp(-T / S(T3)) + S(a) * exp(-T / S(T1)) + exp(-S(T2) / T);
  S L = log10_(Fcent);
  S c = S(-0.4) - S(ORACLE_PLANT == 7 ? -0.67 : 0.67) * L;  // plant 7
  S n = S(0.75) - S(ORACLE_PLANT == 11 ? -1.27 : 1.27) * L;  // plant 11
  S x10 = log10_(Pr);
  S den = n - S(ORACLE_PLANT == 12 ? -0.14 : 0.14) * (x10 + c);  // plant 12
  S f1 = (x10 + c) / den;
  S log10F = L / (S(1.0) + f1 * f1);
  F = pow10_(log10F);
  // d f1 / d log10 Pr = n / den^2;  d log10F / d f1 = -2 L f1 / (1 + f1^2)^2
  dlog10F_dlog10Pr = -S(2.0) * L * f1 / ((S(1.0) + f1 * f1) * (S(1.0) + f1 * f1)) * (n / (den * den));
}

template <class S>
static void rates(const Mech& m, double p, const S* phi, S* f, RateState<S>& st, const S* lnA_shift = nullptr) {
  const int K = m.K, R = m.R;
  st.T = phi[0];
  st.Y.resize(K);
  S ysum = S(0.0);
  for (int k = 0; k < K - 1; ++k) { st.Y[k] = phi[1 + k]; ysum += st.Y[k]; }
  st.Y[K - 1] = S(1.0) - ysum;
  S inv_wbar = S(0.0);
  for (int k = 0; k < K; ++k) inv_wbar += st.Y[k] / S(m.W[k]);
  st.Wbar = S(1.0) / inv_wbar;
  st.rho = S(p) * st.Wbar / (S(kRu) * st.T);
  st.C.resize(K);
  for (int k = 0; k < K; ++k) st.C[k] = st.rho * st.Y[k] / S(m.W[k]);
  thermo(m, st.T, st.th);
  S lnT = log(st.T);
  S invT = S(1.0) / st.T;
  S ln_patm_rut = log(S(kPatm) / (S(kRu) * st.T));
  st.kf.assign(R, S(0.0)); st.kr.assign(R, S(0.0)); st.M.assign(R, S(0.0));
  st.qf.assign(R, S(0.0)); st.qr.assign(R, S(0.0)); st.q.assign(R, S(0.0));
  st.Pr.assign(R, S(0.0)); st.F.assign(R, S(1.0)); st.dlogF_dlogPr.assign(R, S(0.0));
  st.k0.assign(R, S(0.0)); st.kinf.assign(R, S(0.0));
  for (int r = 0; r < R; ++r) {
    const Reaction& x = m.rx[r];
    S lnA = S(std::log(x.A));
    if (lnA_shift) lnA = lnA + lnA_shift[r];  // perturbation of ln A_r (sensitivity runs)
    S kf = exp(lnA + S(x.b) * lnT - S(x.Ea / kRc) * invT);
    S M = S(0.0);
    if (x.type >= 1) {
      for (int k = 0; k < K; ++k) M += S(ORACLE_PLANT == 9 ? 1.0 : x.eff[k]) * st.C[k];  // plant 9
    }
    if (x.type >= 2) {
      S k0 = exp(S(std::log(x.A0)) + S(x.b0) * lnT - S(x.Ea0 / kRc) * invT);
      S Pr = k0 * M / kf;
      S F, dl;
      troe_F(x, st.T, Pr, F, dl);
      st.k0[r] = k0; st.kinf[r] = kf; st.Pr[r] = Pr; st.F[r] = F; st.dlogF_dlogPr[r] = dl;
      kf = kf * Pr / (S(1.0) + Pr) * F;
    }
    // ln Kc = -sum_k nu_k g_k/RT + (sum_k nu_k) ln(Patm/(Ru T))
    S dG_RT = S(0.0);
    int dnu = 0;
    for (int s = 0; s < 2; ++s) {
      if (x.prod[s] >= 0) { dG_RT += st.th.h_RT[x.prod[s]] - st.th.s_R[x.prod[s]]; dnu += 1; }
      if (x.reac[s] >= 0) { dG_RT -= st.th.h_RT[x.reac[s]] - st.th.s_R[x.reac[s]]; dnu -= 1; }
    }
    S Kc = exp(-dG_RT + S((double)(ORACLE_PLANT == 1 ? -dnu : dnu)) * ln_patm_rut);  // plant 1
    S kr = kf / Kc;
    S pf = S(1.0), pr = S(1.0);
    for (int s = 0; s < 2; ++s) {
      if (x.reac[s] >= 0) pf *= st.C[x.reac[s]];
      if (x.prod[s] >= 0) pr *= st.C[x.prod[s]];
    }
    S qf = kf * pf, qr = kr * pr;
    if (x.type == 1) { qf *= M; if (ORACLE_PLANT != 5) qr *= M; }  // plant 5
    st.kf[r] = kf; st.kr[r] = kr; st.M[r] = M; st.qf[r] = qf; st.qr[r] = qr; st.q[r] = qf - qr;
  }
  st.omega.assign(K, S(0.0));
  for (int k = 0; k < K; ++k)
    for (int r = 0; r < R; ++r)
      if (m.nu[k][r] != 0) st.omega[k] += S((double)m.nu[k][r]) * st.q[r];
  st.cp_mass = S(0.0);
  for (int k = 0; k < K; ++k) st.cp_mass += st.Y[k] * st.th.cp_R[k] * S(kRu) / S(m.W[k]);
  S Q = S(0.0);  // sum_k H_k omega_k, erg/(cm^3 s)
  for (int k = 0; k < K; ++k) Q += st.th.h_RT[k] * S(kRu) * st.T * st.omega[k];
  f[0] = (ORACLE_PLANT == 3 ? Q : -Q) / (st.rho * st.cp_mass);  // plant 3
  for (int k = 0; k < K - 1; ++k) f[1 + k] = S(ORACLE_PLANT == 2 ? 1.0 : m.W[k]) * st.omega[k] / st.rho;  // plant 2
}

// ----------------------------------------------------------------------------------------------
// Analytical Jacobian J[i][j] = d f_i / d phi_j, phi = [T, Y_1..Y_{K-1}] (Sec. 2.3).
//
// Chain rule through the concentrations C_j = rho Y_j / W_j, rho = p Wbar/(Ru T),
// Y_K = 1 - sum_{i<K} Y_i:
//   d ln rho / dT = -1/T,   d ln rho / dY_i = -Wbar (1/W_i - 1/W_K)
//   dC_j / dY_i = (rho/W_j)(delta_ij - delta_jK) + C_j d ln rho/dY_i,   dC_j/dT = -C_j/T
// Per reaction: dq/dC_j (mass action, plus efficiencies through [M]), dq/dT at fixed C.
// Then with Z_kj = d omega_k / dC_j and Q = sum_k H_k omega_k:
//   d omega_k/dY_i = (rho/W_i) Z_ki - (rho/W_K) Z_kK + (sum_j Z_kj C_j) d ln rho/dY_i
//   d omega_k/dT   = d omega_k/dT|_C - (1/T) sum_j Z_kj C_j
//   f_Yk = W_k omega_k / rho   ->  d f_Yk/dx = (W_k/rho) d omega_k/dx - f_Yk d ln rho/dx
//   f_T  = -Q/(rho cp)         ->  d f_T/dx  = -(dQ/dx)/(rho cp) - f_T (d ln rho/dx + d ln cp/dx)
//   dQ/dT = sum_k (cp_k omega_k + H_k d omega_k/dT),  dQ/dY_i = sum_k H_k d omega_k/dY_i
//   d cp/dY_i = cp_i/W_i - cp_K/W_K (molar cp_k),  d cp/dT = sum_k Y_k (d cp_k/dT)/W_k

template <class S>
static void jacobian(const Mech& m, double p, const S* phi, S* f, S* J, const S* lnA_shift = nullptr) {
  const int K = m.K, R = m.R, N = K, d = K - 1;
  RateState<S> st;
  rates(m, p, phi, f, st, lnA_shift);
  const S T = st.T, invT = S(1.0) / T;
  std::vector<S> dlnrho_dY(K - 1);
#if ORACLE_PLANT == 6
  for (int i = 0; i < K - 1; ++i) dlnrho_dY[i] = st.Wbar * (S(1.0) / S(m.W[i]) - S(1.0) / S(m.W[d]));  // plant 6
#else
  for (int i = 0; i < K - 1; ++i) dlnrho_dY[i] = -st.Wbar * (S(1.0) / S(m.W[i]) - S(1.0) / S(m.W[d]));
#endif
  // Z = d omega / dC (K x K), and dw/dT at fixed C
  std::vector<S> Z((size_t)K * K, S(0.0)), domega_dT(K, S(0.0));
  std::vector<S> dqdC(K);
  for (int r = 0; r < R; ++r) {
    const Reaction& x = m.rx[r];
    for (int j = 0; j < K; ++j) dqdC[j] = S(0.0);
    // mass-action part: d(prod C)/dC_j by the product rule over the two slots
    auto slot_deriv = [&](const int* sp, const S& kcoef) {
      if (sp[0] >= 0 && sp[1] >= 0) {
        dqdC[sp[0]] += kcoef * st.C[sp[1]];
        dqdC[sp[1]] += kcoef * st.C[sp[0]];
      } else if (sp[0] >= 0) {
        dqdC[sp[0]] += kcoef;
      } else if (sp[1] >= 0) {
        dqdC[sp[1]] += kcoef;
      }
    };
    S pf = S(1.0), pr = S(1.0);
    for (int s = 0; s < 2; ++s) {
      if (x.reac[s] >= 0) pf *= st.C[x.reac[s]];
      if (x.prod[s] >= 0) pr *= st.C[x.prod[s]];
    }
    S mfac = (x.type == 1) ? st.M[r] : S(1.0);
    slot_deriv(x.reac, mfac * st.kf[r]);
    slot_deriv(x.prod, -(mfac * st.kr[r]));
    // d ln kf/dT and d ln Kc/dT at fixed C
    S dlnkf_dT = S(x.b) * invT + S(x.Ea / kRc) * invT * invT;
    S dH_RT = S(0.0);
    int dnu = 0;
    for (int s = 0; s < 2; ++s) {
      if (x.prod[s] >= 0) { dH_RT += st.th.h_RT[x.prod[s]]; dnu += 1; }
      if (x.reac[s] >= 0) { dH_RT -= st.th.h_RT[x.reac[s]]; dnu -= 1; }
    }
    // d(g/RT)/dT = -(h/RT)/T  ->  d ln Kc/dT = (sum nu h/RT)/T - (sum nu)/T
    S dlnKc_dT = (dH_RT - S((double)(ORACLE_PLANT == 1 ? -dnu : dnu))) * invT;  // plant 1
    if (x.type == 1) {
      S R0 = st.kf[r] * pf - st.kr[r] * pr;
      for (int j = 0; j < K; ++j) dqdC[j] += S(x.eff[j]) * R0;
      S dq_dT = st.M[r] * (st.kf[r] * dlnkf_dT * pf - st.kr[r] * (dlnkf_dT - dlnKc_dT) * pr);
      for (int k = 0; k < K; ++k)
        if (m.nu[k][r] != 0) domega_dT[k] += S((double)m.nu[k][r]) * dq_dT;
    } else if (x.type >= 2) {
      // k = kinf Pr/(1+Pr) F(T, Pr), Pr = k0 [M]/kinf
      const S Pr = st.Pr[r], F = st.F[r], k0 = st.k0[r];
      const S dlF = st.dlogF_dlogPr[r];  // d log10 F / d log10 Pr
      // d k/d[M] = k0 F/(1+Pr) (1/(1+Pr) + d log10F/d log10Pr)
      S dk_dM = k0 * F / (S(1.0) + Pr) * (S(1.0) / (S(1.0) + Pr) + dlF);
      S Kc_inv = st.kr[r] / st.kf[r];
      S R1 = pf - Kc_inv * pr;  // q = k (pf - pr/Kc)
      for (int j = 0; j < K; ++j) dqdC[j] += S(x.eff[j]) * dk_dM * R1;
      // d ln k/dT at fixed [M]
      S dlnkinf_dT = dlnkf_dT;
      S dlnk0_dT = S(x.b0) * invT + S(x.Ea0 / kRc) * invT * invT;
      S dlnPr_dT = dlnk0_dT - dlnkinf_dT;
      S dlnF_dT = S(0.0);
      if (x.type == 3) {
        const double a = x.troe[0], T3 = x.troe[1], T1 = x.troe[2], T2 = x.troe[3];
        S e3 = exp(-T / S(T3)), e1 = exp(-T / S(T1)), e2 = exp(-S(T2) / T);
        S Fcent = S(1.0 - a) * e3 + S(a) * e1 + e2;
        S dFcent_dT = -S(1.0 - a) / S(T3) * e3 - S(a) / S(T1) * e1 + S(T2) * invT * invT * e2;
        S L = log10_(Fcent);
        S dL_dT = dFcent_dT / (Fcent * S(std::log(10.0)));
        S c = S(-0.4) - S(ORACLE_PLANT == 7 ? -0.67 : 0.67) * L, n = S(0.75) - S(1.27) * L;  // plant 7
        S x10 = log10_(Pr);
        S den = n - S(0.14) * (x10 + c);
        S f1 = (x10 + c) / den;
        S g = S(1.0) + f1 * f1;
        // d f1 / dL at fixed Pr, with dc/dL = -0.67, dn/dL = -1.27
        const S dc_dL = S(ORACLE_PLANT == 7 ? 0.67 : -0.67);  // plant 7
        S df1_dL = (dc_dL * den - (x10 + c) * (S(-1.27) - S(0.14) * dc_dL)) / (den * den);
        S dlog10F_dL = S(1.0) / g - L * S(2.0) * f1 / (g * g) * df1_dL;
        dlnF_dT = S(std::log(10.0)) * dlog10F_dL * dL_dT;
      }
      S dlnk_dT = dlnkinf_dT + (S(1.0) / (S(1.0) + Pr) + dlF) * dlnPr_dT + dlnF_dT;
      S dq_dT = st.kf[r] * dlnk_dT * pf - st.kr[r] * (dlnk_dT - dlnKc_dT) * pr;
      for (int k = 0; k < K; ++k)
        if (m.nu[k][r] != 0) domega_dT[k] += S((double)m.nu[k][r]) * dq_dT;
    } else {
      S dq_dT = st.kf[r] * dlnkf_dT * pf - st.kr[r] * (dlnkf_dT - dlnKc_dT) * pr;
      for (int k = 0; k < K; ++k)
        if (m.nu[k][r] != 0) domega_dT[k] += S((double)m.nu[k][r]) * dq_dT;
    }
    // species with a non-zero dq/dC: the slot species, or every species when [M] enters q
    std::vector<int> cols;
    if (x.type >= 1) {
      for (int j = 0; j < K; ++j) cols.push_back(j);
    } else {
      for (int s = 0; s < 2; ++s)
        for (int sp : {x.reac[s], x.prod[s]})
          if (sp >= 0 && std::find(cols.begin(), cols.end(), sp) == cols.end()) cols.push_back(sp);
    }
    for (int k = 0; k < K; ++k) {
      if (m.nu[k][r] == 0) continue;
      S nk = S((double)m.nu[k][r]);
      for (int j : cols) Z[(size_t)k * K + j] += nk * dqdC[j];
    }
  }
  // d omega_k / dY_i and d omega_k / dT (total)
  std::vector<S> ZC(K, S(0.0));
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < K; ++j) ZC[k] += Z[(size_t)k * K + j] * st.C[j];
  std::vector<S> dw_dY((size_t)K * (K - 1)), dw_dT(K);
  for (int k = 0; k < K; ++k) {
    for (int i = 0; i < K - 1; ++i)
      dw_dY[(size_t)k * (K - 1) + i] = st.rho / S(m.W[i]) * Z[(size_t)k * K + i] -
                                       st.rho / S(m.W[d]) * Z[(size_t)k * K + d] + ZC[k] * dlnrho_dY[i];
    dw_dT[k] = domega_dT[k] - ZC[k] * invT;
  }
  // species rows
  for (int k = 0; k < K - 1; ++k) {
    const S Wk = S(ORACLE_PLANT == 2 ? 1.0 : m.W[k]);  // plant 2
    J[(size_t)(1 + k) * N + 0] = Wk / st.rho * dw_dT[k] + f[1 + k] * invT;  // -f * dlnrho/dT
    for (int i = 0; i < K - 1; ++i)
      J[(size_t)(1 + k) * N + 1 + i] = Wk / st.rho * dw_dY[(size_t)k * (K - 1) + i] - f[1 + k] * dlnrho_dY[i];
  }
  // temperature row
  const S rhocp = st.rho * st.cp_mass;
  S dQ_dT = S(0.0);
  for (int k = 0; k < K; ++k) {
    S Hk = st.th.h_RT[k] * S(kRu) * T;
    S cpk = st.th.cp_R[k] * S(kRu);
    dQ_dT += cpk * st.omega[k] + Hk * dw_dT[k];
  }
  S dcp_dT = S(0.0);
  for (int k = 0; k < K; ++k) dcp_dT += st.Y[k] * st.th.dcp_RdT[k] * S(kRu) / S(m.W[k]);
#if ORACLE_PLANT == 3
  J[0] = dQ_dT / rhocp - f[0] * (-invT + dcp_dT / st.cp_mass);  // plant 3
#else
  J[0] = -dQ_dT / rhocp - f[0] * (-invT + dcp_dT / st.cp_mass);
#endif
  for (int i = 0; i < K - 1; ++i) {
    S dQ_dYi = S(0.0);
    for (int k = 0; k < K; ++k) dQ_dYi += st.th.h_RT[k] * S(kRu) * T * dw_dY[(size_t)k * (K - 1) + i];
    S dcp_dYi = st.th.cp_R[i] * S(kRu) / S(m.W[i]) - st.th.cp_R[d] * S(kRu) / S(m.W[d]);
#if ORACLE_PLANT == 3
    J[1 + i] = dQ_dYi / rhocp - f[0] * (dlnrho_dY[i] + dcp_dYi / st.cp_mass);  // plant 3
#else
    J[1 + i] = -dQ_dYi / rhocp - f[0] * (dlnrho_dY[i] + dcp_dYi / st.cp_mass);
#endif
  }
#if ORACLE_PLANT == 10
  // plant 10: the Jacobian returned transposed
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) std::swap(J[(size_t)i * N + j], J[(size_t)j * N + i]);
#endif
}

// ----------------------------------------------------------------------------------------------
// First-order forward-difference Jacobian: the alternative the paper measures the analytical
// Jacobian against (Sec. 2.3; "first-order finite differencing", N + 1 rate evaluations).
// Column j = (f(phi + d_j e_j) - f(phi)) / d_j, d_j = 2^-26 max(|phi_j|, s_j), s_0 = 1 K for T and
// s_j = 1e-6 for the mass fractions; f0 = f(phi) on return.

static void jacobian_fd(const Mech& m, double p, const double* phi, double* f0, double* J) {
  const int N = m.K;
  RateState<double> st;
  rates(m, p, phi, f0, st);
  std::vector<double> x(phi, phi + N), fj(N);
  for (int j = 0; j < N; ++j) {
    const double d = 0x1p-26 * std::max(std::fabs(phi[j]), j == 0 ? 1.0 : 1e-6);
    x[j] = phi[j] + d;
    const double dj = x[j] - phi[j];  // the step actually taken
    RateState<double> sj;
    rates(m, p, x.data(), fj.data(), sj);
    for (int i = 0; i < N; ++i) J[(size_t)i * N + j] = (fj[i] - f0[i]) / dj;
    x[j] = phi[j];
  }
}

// ----------------------------------------------------------------------------------------------
// Dense LU with partial pivoting (textbook Doolittle, row interchanges; ties go to the lowest
// row index) and the forward / back substitution that uses it.

template <class S>
static bool lu_factor(int n, S* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::abs(re(a[(size_t)k * n + k]));
    for (int i = k + 1; i < n; ++i) {
      double v = std::abs(re(a[(size_t)i * n + k]));
      if (v > best) { best = v; p = i; }
    }
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(a[(size_t)k * n + j], a[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      a[(size_t)i * n + k] = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      for (int j = k + 1; j < n; ++j) a[(size_t)i * n + j] -= a[(size_t)i * n + k] * a[(size_t)k * n + j];
    }
  }
  return true;
}

template <class S>
static void lu_solve(int n, const S* a, const int* piv, S* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[(size_t)i * n + j] * b[j];
    b[i] = b[i] / a[(size_t)i * n + i];
  }
}

// ----------------------------------------------------------------------------------------------
// Rosenbrock method, classical form (Hairer & Wanner, Solving ODEs II, Sec. IV.7):
//   (I - gamma h J) k_i = h f(y + sum_{j<i} alpha_ij k_j) + h J sum_{j<i} gamma_ij k_j
//   y_new = y + sum b_i k_i,   error = sum (b_i - bhat_i) k_i
// 4 stages, order 4, embedded order 3, L-stable (R(inf) = 0), R_hat(inf) = 1/2.  gamma is the
// root near 0.5728 of the order-4 L-stability polynomial; alpha_21 = 2 gamma, alpha_3 = alpha_4
// = 0.65 (stage 4 reuses stage 3's argument), b_3 = 0, beta_43 = -0.23.  The remaining
// coefficients solve the order conditions exactly (checked by the tests).

struct Ros4 {
  static constexpr int s = 4;
  double gamma = 0.5728160624821348554080014;
  double alpha[4][4] = {{0, 0, 0, 0},
                        {1.145632124964269710816, 0, 0, 0},
                        {0.5153579993305085683839, 0.1346420006694914316161, 0, 0},
                        {0.5153579993305085683839, 0.1346420006694914316161, 0.0, 0}};
  double gam[4][4] = {{0, 0, 0, 0},
                      {-2.341993140193055730037, 0, 0, 0},
                      {-0.02787068958553465628054, 0.2086236229782045434317, 0, 0},
                      {-0.2474922550210316401721, -0.1907869111079863467924, -0.23, 0}};
  double b[4] = {0.3189845243949336284427 + (ORACLE_PLANT == 8 ? 1e-3 : 0.0),  // plant 8
                 0.05124233729027201389922, 0.0, 0.6297731383147943576581};
  double bhat[4] = {0.04912862293304546304649, -0.07686730508695069897692, -0.1719498044983180858675,
                    1.199688486652223321798};
};

enum Status { kOk = 0, kMaxSteps = 1, kHUnderflow = 2, kBadInput = 3 };

struct CellStats {
  int64_t steps = 0, rejects = 0, f_evals = 0, lu = 0;
};

// Step-size controller (paper Sec. 2.3: adaptive sub-steps under rtol/atol; formula from
// Hairer & Wanner IV.8):  e = (I - gamma h J)^-1 sum (b_i - bhat_i) k_i (filtered estimate),
// err = max_i |e_i| / (atol + rtol max(|y_i|, |ynew_i|));
// accept if err <= 1; h_new = h min(facmax, max(0.2, 0.9 err^(-1/4))), facmax = 6, or 1 on the
// step after a rejection.  Non-finite err or a singular pivot counts as a rejection with factor
// 0.2.  The last step is clipped so that t reaches dt exactly.  The cold-start step is
// 0.01 dt; a positive h_inout overrides it (carry-over of the chemistry sub-step, Sec. 2.3).
static int integrate_cell(const Mech& m, double p, double* phi, double dt, double rtol, double atol, double* h_io,
                          int max_steps, CellStats& cs, std::vector<double>* h_record = nullptr,
                          bool fd_jacobian = false) {
  const int N = m.K;
  if (!(std::isfinite(phi[0]) && phi[0] > 0.0)) return kBadInput;
  for (int i = 1; i < N; ++i)
    if (!std::isfinite(phi[i])) return kBadInput;
  Ros4 c;
  std::vector<double> y(phi, phi + N), ynew(N), f0(N), fi(N), J((size_t)N * N), A((size_t)N * N), yi(N), g(N),
      rhs(N), err(N);
  std::vector<std::vector<double>> k(4, std::vector<double>(N));
  std::vector<int> piv(N);
  double h = (h_io && *h_io > 0.0) ? std::min(*h_io, dt) : 0.01 * dt;
  double t = 0.0;
  bool need_jac = true, last_rejected = false;
  double h_next_unclipped = h;
  int status = kOk;
  for (int attempt = 0;; ++attempt) {
    if (attempt >= max_steps) { status = kMaxSteps; break; }
    if (h_next_unclipped < 1e-14 * dt) { status = kHUnderflow; break; }
    if (need_jac) {
      if (fd_jacobian) {
        jacobian_fd(m, p, y.data(), f0.data(), J.data());
        cs.f_evals += N + 1;
      } else {
        jacobian(m, p, y.data(), f0.data(), J.data());
        cs.f_evals++;
      }
      need_jac = false;
    }
    for (size_t e = 0; e < (size_t)N * N; ++e) A[e] = -c.gamma * h * J[e];
    for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += 1.0;
    bool ok = lu_factor(N, A.data(), piv.data());
    cs.lu++;
    double errn = INFINITY;
    if (ok) {
      for (int s = 0; s < 4; ++s) {
        for (int i = 0; i < N; ++i) {
          yi[i] = y[i];
          g[i] = 0.0;
          for (int j = 0; j < s; ++j) { yi[i] += c.alpha[s][j] * k[j][i]; g[i] += c.gam[s][j] * k[j][i]; }
        }
        if (s == 0) {
          fi = f0;
        } else {
          RateState<double> st;
          rates(m, p, yi.data(), fi.data(), st);
          cs.f_evals++;
        }
        for (int i = 0; i < N; ++i) {
          double jg = 0.0;
          for (int j = 0; j < N; ++j) jg += J[(size_t)i * N + j] * g[j];
          rhs[i] = h * fi[i] + h * jg;
        }
        lu_solve(N, A.data(), piv.data(), rhs.data());
        k[s] = rhs;
      }
      for (int i = 0; i < N; ++i) {
        double yn = y[i], e = 0.0;
        for (int s = 0; s < 4; ++s) { yn += c.b[s] * k[s][i]; e += (c.b[s] - c.bhat[s]) * k[s][i]; }
        ynew[i] = yn;
        err[i] = e;
      }
      // error filter: the embedded difference is passed through (I - gamma h J)^-1, which leaves
      // non-stiff components unchanged and damps stiff ones, whose raw estimate does not shrink
      // with h because R_hat(inf) != 0 (Shampine; Hairer & Wanner IV.8)
      lu_solve(N, A.data(), piv.data(), err.data());
      errn = 0.0;
      for (int i = 0; i < N; ++i) {
        double sc = atol + rtol * std::max(std::fabs(y[i]), std::fabs(ynew[i]));
        double r = std::fabs(err[i]) / sc;
        if (!(r <= errn)) errn = r;  // propagates NaN
      }
    }
    double fac;
    if (std::isfinite(errn) && errn <= 1.0) {
      if (h_record) h_record->push_back(h);
      t = (h >= dt - t) ? dt : t + h;
      y = ynew;
      cs.steps++;
      need_jac = true;
      fac = std::min(6.0, std::max(0.2, 0.9 * std::pow(errn, -0.25)));
      if (last_rejected) fac = std::min(fac, 1.0);
      last_rejected = false;
      h_next_unclipped = h * fac;
      if (t >= dt) break;
    } else {
      cs.rejects++;
      fac = std::isfinite(errn) ? std::max(0.2, 0.9 * std::pow(errn, -0.25)) : 0.2;
      fac = std::min(fac, 1.0);
      last_rejected = true;
      h_next_unclipped = h * fac;
    }
    h = std::min(h_next_unclipped, dt - t);
  }
  for (int i = 0; i < N; ++i) phi[i] = y[i];
  if (h_io) *h_io = h_next_unclipped;
  return status;
}

// ----------------------------------------------------------------------------------------------
// Seulex: the linearly implicit Euler method with extrapolation (the paper's integrator,
// Sec. 2.3, following Hairer & Wanner, Solving ODEs II, Sec. IV.9).  One macro step of size H
// from y, with J = J(y):
//   column j = 1..: n_j = j sub-steps of h = H/n_j,  (I - h J)(y_{i+1} - y_i) = h f(y_i),
//   T_{j,1} = y_{n_j};  T_{j,l} = T_{j,l-1} + (T_{j,l-1} - T_{j-1,l-1}) / (n_j/n_{j-l+1} - 1)
//   err_j = max_i |T_{j,j} - T_{j,j-1}| / (atol + rtol max(|y_i|, |T_{j,j,i}|)),
//   fac_j = min(4, max(0.02, 0.94 err_j^(-1/j))).
// With target column k (2 <= k <= kmax-1) the columns up to k+1 are computed as needed:
//   j = k-1 (j >= 2): accept if err <= 1;
//   j = k:            accept if err <= 1; give up if err > (n_{k+1} / n_1)^2;
//   j = k+1:          accept if err <= 1, else give up.
// (Column k-1 never gives up early: on linear test problems at tight tolerances a give-up there
// predicted from the square of the step-number ratio rejected steps that column k accepts, and
// the controller cycled at low order.)
// Accepted at column c: y <- T_{c,c}; the next target and step minimise the work per unit step
// w_j = A_j / (H fac_j), A_j the cost of columns 1..j in rate-evaluation units (Jacobian 2.5,
// LU 2, rate evaluation 1, solve 0.2):
//   c = 2:      k = 3, H <- H fac_2 A_3/A_2 (H fac_2 after a rejection);
//   2 < c <= k: k = c, or c-1 if w_{c-1} < 0.8 w_c, or c+1 if c = k and w_c < 0.9 w_{c-1};
//               H <- H fac_min(k,c) (times A_k/A_c when k > c);
//   c = k+1:    k = c-1, or c if w_c < 0.9 w_{c-1}; H <- H fac_k;
//   after a rejection H does not grow and k <= c.
// Given up: H <- H min(fac_m, 1/2) with m = min(k, last column), k <- m (J is kept).  A singular
// iteration matrix or a non-finite error gives up with H <- H/5.  Cold start H = 0.01 dt, k = 2.
// The last step is clipped to end at dt; h_inout carries the unclipped proposal over.
struct Seulex {
  static constexpr int kmax = 8;
  double A[kmax + 1];
  Seulex() {
    const double cJ = 2.5, cLU = 2.0, cf = 1.0, cs = 0.2;
    A[0] = 0.0;
    A[1] = cJ + cLU + 1.0 * (cs + cf);
    for (int j = 2; j <= kmax; ++j) A[j] = A[j - 1] + cLU + j * cs + (j - 1) * cf;
  }
  static int n(int j) { return j; }
};

static int integrate_cell_seulex(const Mech& m, double p, double* phi, double dt, double rtol, double atol,
                                 double* h_io, int max_steps, CellStats& cs) {
  const int N = m.K;
  if (!(std::isfinite(phi[0]) && phi[0] > 0.0)) return kBadInput;
  for (int i = 1; i < N; ++i)
    if (!std::isfinite(phi[i])) return kBadInput;
  Seulex c;
  const int kmax = Seulex::kmax;
  std::vector<double> y(phi, phi + N), f0(N), fi(N), yi(N), d(N), J((size_t)N * N), W((size_t)N * N), q(N),
      qn(N);
  std::vector<std::vector<double>> T(kmax + 1, std::vector<double>(N));  // T[l] = current row's T_{.,l}
  std::vector<int> piv(N);
  double H = (h_io && *h_io > 0.0) ? std::min(*h_io, dt) : 0.01 * dt;
  double t = 0.0, H_next_unclipped = H;
  int k = 2;
  bool need_jac = true, last_rejected = false;
  int status = kOk;
  for (int attempt = 0;; ++attempt) {
    if (attempt >= max_steps) { status = kMaxSteps; break; }
    if (H_next_unclipped < 1e-14 * dt) { status = kHUnderflow; break; }
    if (need_jac) {
      jacobian(m, p, y.data(), f0.data(), J.data());
      cs.f_evals++;
      need_jac = false;
    }
    double err[kmax + 2], fac[kmax + 2];
    int accepted = 0, last = 0;
    bool bad = false;
    for (int j = 1; j <= k + 1; ++j) {
      last = j;
      const double h = H / Seulex::n(j);
      for (size_t e = 0; e < (size_t)N * N; ++e) W[e] = -h * J[e];
      for (int i = 0; i < N; ++i) W[(size_t)i * N + i] += 1.0;
      cs.lu++;
      if (!lu_factor(N, W.data(), piv.data())) { bad = true; break; }
      yi = y;
      for (int s = 0; s < Seulex::n(j); ++s) {
        if (s == 0) {
          fi = f0;
        } else {
          RateState<double> st;
          rates(m, p, yi.data(), fi.data(), st);
          cs.f_evals++;
        }
        for (int i = 0; i < N; ++i) d[i] = h * fi[i];
        lu_solve(N, W.data(), piv.data(), d.data());
        for (int i = 0; i < N; ++i) yi[i] += d[i];
      }
      // Aitken-Neville: T holds row j-1 in T[1..j-1]; build row j, overwriting as we go
      q = yi;
      for (int l = 2; l <= j; ++l) {
        const double r = (double)Seulex::n(j) / (double)Seulex::n(j - l + 1);
        for (int i = 0; i < N; ++i) qn[i] = q[i] + (q[i] - T[l - 1][i]) / (r - 1.0);
        T[l - 1] = q;
        q = qn;
      }
      T[j] = q;
      if (j < 2) continue;
      double e = 0.0;
      for (int i = 0; i < N; ++i) {
        const double sc = atol + rtol * std::max(std::fabs(y[i]), std::fabs(T[j][i]));
        const double r = std::fabs(T[j][i] - T[j - 1][i]) / sc;
        if (!(r <= e)) e = r;  // propagates NaN
      }
      if (!std::isfinite(e)) { bad = true; break; }
      err[j] = e;
      fac[j] = (e > 0.0) ? std::min(4.0, std::max(0.02, 0.94 * std::pow(e, -1.0 / j))) : 4.0;
      const double n1 = Seulex::n(1), nk1 = Seulex::n(k + 1);
      if (j == k - 1) {
        if (e <= 1.0) { accepted = j; break; }
      } else if (j == k) {
        if (e <= 1.0) { accepted = j; break; }
        if (e > (nk1 / n1) * (nk1 / n1)) break;
      } else if (j == k + 1) {
        if (e <= 1.0) accepted = j;
        break;
      }
    }
    if (accepted) {
      const int a = accepted;
      t = (H >= dt - t) ? dt : t + H;
      y = T[a];
      cs.steps++;
      need_jac = true;
      auto w = [&](int j) { return c.A[j] / (H * fac[j]); };
      int knew;
      double Hn;
      if (a == 2) {
        knew = 3;
        Hn = H * fac[2] * (last_rejected ? 1.0 : c.A[3] / c.A[2]);
      } else if (a <= k) {
        knew = a;
        if (w(a - 1) < 0.8 * w(a)) knew = a - 1;
        else if (a == k && w(a) < 0.9 * w(a - 1)) knew = a + 1;
        Hn = H * fac[std::min(knew, a)] * (knew > a ? c.A[knew] / c.A[a] : 1.0);
      } else {
        knew = a - 1;
        if (w(a) < 0.9 * w(a - 1)) knew = a;
        Hn = H * fac[knew];
      }
      if (last_rejected) { Hn = std::min(Hn, H); knew = std::min(knew, a); }
      k = std::max(2, std::min(knew, kmax - 1));
      last_rejected = false;
      H_next_unclipped = Hn;
      if (t >= dt) break;
    } else {
      cs.rejects++;
      last_rejected = true;
      if (bad) {
        H_next_unclipped = H * 0.2;
      } else {
        const int mcol = std::min(k, last);
        H_next_unclipped = H * std::min(fac[mcol], 0.5);
        k = std::max(2, mcol);
      }
    }
    H = std::min(H_next_unclipped, dt - t);
  }
  for (int i = 0; i < N; ++i) phi[i] = y[i];
  if (h_io) *h_io = H_next_unclipped;
  return status;
}

// One Rosenbrock step of size h from y (no error control): the same classical-form formulas as
// integrate_cell, templated so that the dual-number instance gives the tangent-linear step
// (forward sensitivities through the discrete method with the step size frozen).
template <class S>
static bool ros_step(const Mech& m, double p, std::vector<S>& y, double h, const S* lnA_shift) {
  const int N = m.K;
  Ros4 c;
  std::vector<S> f0(N), fi(N), J((size_t)N * N), A((size_t)N * N), yi(N), g(N), rhs(N);
  std::vector<std::vector<S>> k(4, std::vector<S>(N));
  std::vector<int> piv(N);
  jacobian(m, p, y.data(), f0.data(), J.data(), lnA_shift);
  for (size_t e = 0; e < (size_t)N * N; ++e) A[e] = -S(c.gamma * h) * J[e];
  for (int i = 0; i < N; ++i) A[(size_t)i * N + i] += S(1.0);
  if (!lu_factor(N, A.data(), piv.data())) return false;
  for (int s = 0; s < 4; ++s) {
    for (int i = 0; i < N; ++i) {
      yi[i] = y[i];
      g[i] = S(0.0);
      for (int j = 0; j < s; ++j) { yi[i] += S(c.alpha[s][j]) * k[j][i]; g[i] += S(c.gam[s][j]) * k[j][i]; }
    }
    if (s == 0) {
      fi = f0;
    } else {
      RateState<S> st;
      rates(m, p, yi.data(), fi.data(), st, lnA_shift);
    }
    for (int i = 0; i < N; ++i) {
      S jg = S(0.0);
      for (int j = 0; j < N; ++j) jg += J[(size_t)i * N + j] * g[j];
      rhs[i] = S(h) * fi[i] + S(h) * jg;
    }
    lu_solve(N, A.data(), piv.data(), rhs.data());
    k[s] = rhs;
  }
  for (int i = 0; i < N; ++i)
    for (int s = 0; s < 4; ++s) y[i] += S(c.b[s]) * k[s][i];
  return true;
}

}  // namespace oracle

// ==============================================================================================
// C interface for the tests and the benchmark's CPU baseline.

using namespace oracle;

static thread_local std::string g_err;

extern "C" {

const char* oracle_last_error() { return g_err.c_str(); }

void* oracle_load(const char* path) {
  Mech* m = new Mech();
  if (!load_mech(path, *m, g_err)) { delete m; return nullptr; }
  return m;
}

void oracle_free(void* h) { delete static_cast<Mech*>(h); }

// The oracle's reading of the mechanism, in the text form of the library's
// chem_describe_mechanism (species "sp W Tmid a_low a_high", reactions "rx type n_reac reac..
// n_prod prod.. A b Ea/R [eff ..] [low A0 b0 Ea0/R] [troe alpha T3 T1 T2]"), so that tests can
// compare the two independent readers.  *need = size with the NUL; cap <= 0 only queries it.
int oracle_describe(void* h, char* buf, int64_t cap, int64_t* need) {
  const Mech* m = static_cast<const Mech*>(h);
  std::ostringstream o;
  o.precision(17);
  o << "species " << m->K << "\n";
  for (int k = 0; k < m->K; ++k) {
    o << "sp " << m->W[k] << " " << m->Tmid[k];
    for (double a : m->alow[k]) o << " " << a;
    for (double a : m->ahigh[k]) o << " " << a;
    o << "\n";
  }
  o << "reactions " << m->R << "\n";
  for (const Reaction& x : m->rx) {
    o << "rx " << x.type;
    for (const int* side : {x.reac, x.prod}) {
      std::vector<int> sp;
      for (int i = 0; i < 2; ++i)
        if (side[i] >= 0) sp.push_back(side[i]);
      std::sort(sp.begin(), sp.end());
      o << " " << sp.size();
      for (int k : sp) o << " " << k;
    }
    o << " " << x.A << " " << x.b << " " << x.Ea / kRc;
    if (x.type >= 1) {
      o << " eff";
      for (double e : x.eff) o << " " << e;
    }
    if (x.type >= 2) o << " low " << x.A0 << " " << x.b0 << " " << x.Ea0 / kRc;
    if (x.type == 3) o << " troe " << x.troe[0] << " " << x.troe[1] << " " << x.troe[2] << " " << x.troe[3];
    o << "\n";
  }
  const std::string t = o.str();
  *need = (int64_t)t.size() + 1;
  if (cap <= 0) return 0;
  if (cap < *need) return 1;
  std::memcpy(buf, t.c_str(), t.size() + 1);
  return 0;
}

int oracle_dims(void* h, int* K, int* R) {
  Mech* m = static_cast<Mech*>(h);
  *K = m->K; *R = m->R;
  return 0;
}

// Species thermo at one temperature: cp/R, h/RT, s/R (K each).
int oracle_thermo(void* h, double T, double* cp_R, double* h_RT, double* s_R) {
  Mech* m = static_cast<Mech*>(h);
  Thermo<double> th;
  thermo(*m, T, th);
  for (int k = 0; k < m->K; ++k) { cp_R[k] = th.cp_R[k]; h_RT[k] = th.h_RT[k]; s_R[k] = th.s_R[k]; }
  return 0;
}

// d/dT of h/RT*T (=h/R) and s/R by complex step, for the thermo consistency pins.
int oracle_thermo_cs(void* h, double T, double step, double* dhR_dT, double* dsR_dT) {
  Mech* m = static_cast<Mech*>(h);
  using C = std::complex<double>;
  Thermo<C> th;
  C Tc(T, step);
  thermo(*m, Tc, th);
  for (int k = 0; k < m->K; ++k) {
    dhR_dT[k] = (th.h_RT[k] * Tc).imag() / step;
    dsR_dT[k] = th.s_R[k].imag() / step;
  }
  return 0;
}

// f for n cells.  p in Pa.  T[n], Y[K][n] species-major (all K species; Y_K is recomputed
// from the others as in Eq. 1), out f[N][n].  Optional per-cell gross scale
// gross[N][n] = |.| sums of the forward and reverse fluxes entering each component.
int oracle_rates(void* h, double p_Pa, int64_t n, const double* T, const double* Y, double* f, double* gross) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K, N = K;
  const double p = p_Pa * 10.0;
  std::vector<double> phi(N), fo(N);
  for (int64_t c = 0; c < n; ++c) {
    phi[0] = T[c];
    for (int k = 0; k < K - 1; ++k) phi[1 + k] = Y[(size_t)k * n + c];
    RateState<double> st;
    rates(*m, p, phi.data(), fo.data(), st);
    for (int i = 0; i < N; ++i) f[(size_t)i * n + c] = fo[i];
    if (gross) {
      std::vector<double> gk(K, 0.0);
      double gT = 0.0;
      for (int r = 0; r < m->R; ++r)
        for (int k = 0; k < K; ++k)
          if (m->nu[k][r] != 0) {
            double a = std::abs((double)m->nu[k][r]) * (std::fabs(st.qf[r]) + std::fabs(st.qr[r]));
            gk[k] += a;
            gT += std::fabs(st.th.h_RT[k] * kRu * st.T) * a;
          }
      gross[c] = gT / (st.rho * st.cp_mass);
      for (int k = 0; k < K - 1; ++k) gross[(size_t)(1 + k) * n + c] = m->W[k] * gk[k] / st.rho;
    }
  }
  return 0;
}

// Per-reaction quantities at one state (tests): kf, kr (effective), qf, qr, and ln Kc.
int oracle_reaction_rates(void* h, double p_Pa, double T, const double* Y, double* kf, double* kr, double* qf,
                          double* qr) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K;
  std::vector<double> phi(K), fo(K);
  phi[0] = T;
  for (int k = 0; k < K - 1; ++k) phi[1 + k] = Y[k];
  RateState<double> st;
  rates(*m, p_Pa * 10.0, phi.data(), fo.data(), st);
  for (int r = 0; r < m->R; ++r) { kf[r] = st.kf[r]; kr[r] = st.kr[r]; qf[r] = st.qf[r]; qr[r] = st.qr[r]; }
  return 0;
}

// Analytical Jacobian for n cells: J[n][N][N], row i = d f_i.
int oracle_jacobian(void* h, double p_Pa, int64_t n, const double* T, const double* Y, double* J) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K, N = K;
  std::vector<double> phi(N), fo(N);
  for (int64_t c = 0; c < n; ++c) {
    phi[0] = T[c];
    for (int k = 0; k < K - 1; ++k) phi[1 + k] = Y[(size_t)k * n + c];
    jacobian(*m, p_Pa * 10.0, phi.data(), fo.data(), J + (size_t)c * N * N);
  }
  return 0;
}

// Directional derivatives at one state phi (N): f and J (row i = d f_i / d phi) together with
// their derivatives df, dJ along (dphi, dlnA) (dual numbers; either direction may be NULL).
int oracle_jacobian_dir(void* h, double p_Pa, const double* phi, const double* dphi, const double* dlnA, double* f,
                        double* J, double* df, double* dJ) {
  Mech* m = static_cast<Mech*>(h);
  const int N = m->K;
  std::vector<Dual> x(N), fo(N), Jd((size_t)N * N), shift(m->R);
  for (int i = 0; i < N; ++i) x[i] = Dual(phi[i], dphi ? dphi[i] : 0.0);
  for (int r = 0; r < m->R; ++r) shift[r] = Dual(0.0, dlnA ? dlnA[r] : 0.0);
  jacobian(*m, p_Pa * 10.0, x.data(), fo.data(), Jd.data(), shift.data());
  for (int i = 0; i < N; ++i) { f[i] = fo[i].v; df[i] = fo[i].d; }
  for (size_t e = 0; e < (size_t)N * N; ++e) { J[e] = Jd[e].v; dJ[e] = Jd[e].d; }
  return 0;
}

// Forward-difference Jacobian of f at one state phi (N): J[N][N] (row i = d f_i / d phi).
int oracle_jacobian_fd(void* h, double p_Pa, const double* phi, double* J) {
  Mech* m = static_cast<Mech*>(h);
  std::vector<double> f0(m->K);
  jacobian_fd(*m, p_Pa * 10.0, phi, f0.data(), J);
  return 0;
}

// Complex-step Jacobian of f at one state: Jcs[N][N] with Jcs[i][j] = Im f_i(phi + i h e_j)/h.
int oracle_jacobian_cs(void* h, double p_Pa, double T, const double* Y, double step, double* Jcs) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K, N = K;
  using C = std::complex<double>;
  std::vector<C> phi(N), fo(N);
  for (int j = 0; j < N; ++j) {
    phi[0] = C(T, 0.0);
    for (int k = 0; k < K - 1; ++k) phi[1 + k] = C(Y[k], 0.0);
    phi[j] += C(0.0, step);
    RateState<C> st;
    rates(*m, p_Pa * 10.0, phi.data(), fo.data(), st);
    for (int i = 0; i < N; ++i) Jcs[(size_t)i * N + j] = fo[i].imag() / step;
  }
  return 0;
}

// Integrate n cells over dt.  T[n] and Y[K][n] are updated in place (Y_K = 1 - sum of the
// others on output).  h_inout[n] may be NULL.  status[n], steps[n], rejects[n] may be NULL.
// solver 0 = Rosenbrock (integrate_cell), 1 = Seulex (integrate_cell_seulex), 2 = Rosenbrock
// with the forward-difference Jacobian.
int oracle_integrate(void* h, double p_Pa, int64_t n, double* T, double* Y, double dt, double rtol, double atol,
                     double* h_inout, int32_t* status, int32_t* steps, int32_t* rejects, int max_steps, int nthreads,
                     int solver) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K, N = K;
  if (nthreads < 1) nthreads = 1;
  std::atomic<int64_t> next(0);
  auto work = [&]() {
    std::vector<double> phi(N);
    for (;;) {
      int64_t c = next.fetch_add(1);
      if (c >= n) break;
      phi[0] = T[c];
      for (int k = 0; k < K - 1; ++k) phi[1 + k] = Y[(size_t)k * n + c];
      CellStats cs;
      int st = (solver == 1)
                   ? integrate_cell_seulex(*m, p_Pa * 10.0, phi.data(), dt, rtol, atol,
                                           h_inout ? &h_inout[c] : nullptr, max_steps, cs)
                   : integrate_cell(*m, p_Pa * 10.0, phi.data(), dt, rtol, atol, h_inout ? &h_inout[c] : nullptr,
                                    max_steps, cs, nullptr, solver == 2);
      T[c] = phi[0];
      double ysum = 0.0;
      for (int k = 0; k < K - 1; ++k) { Y[(size_t)k * n + c] = phi[1 + k]; ysum += phi[1 + k]; }
      Y[(size_t)(K - 1) * n + c] = 1.0 - ysum;
      if (status) status[c] = st;
      if (steps) steps[c] = (int32_t)cs.steps;
      if (rejects) rejects[c] = (int32_t)cs.rejects;
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nthreads; ++t) pool.emplace_back(work);
  work();
  for (auto& th : pool) th.join();
  return 0;
}

// Integrate one cell and return the sizes of its accepted steps (hs[max_hs], *n_hs), for
// replaying the same discrete map.  phi_io = [T, Y_1..Y_{K-1}] in/out.  Returns the status.
int oracle_integrate_record(void* h, double p_Pa, double* phi_io, double dt, double rtol, double atol, double* hs,
                            int max_hs, int* n_hs) {
  Mech* m = static_cast<Mech*>(h);
  std::vector<double> rec;
  CellStats cs;
  int st = integrate_cell(*m, p_Pa * 10.0, phi_io, dt, rtol, atol, nullptr, 100000, cs, &rec);
  *n_hs = (int)rec.size();
  for (int i = 0; i < (int)rec.size() && i < max_hs; ++i) hs[i] = rec[i];
  return st;
}

// Replay the accepted steps hs[0..n) from phi (N) without error control: phi_out = the final
// state, with ln A_r shifted by lnA_shift[r] (R, file order; may be NULL).  With dphi (N) and/or
// dlnA (R) non-NULL, also the tangent-linear result dphi_out = d phi_out along (dphi, dlnA)
// (dual numbers through the same discrete steps).
int oracle_replay(void* h, double p_Pa, const double* phi, const double* hs, int n, const double* lnA_shift,
                  const double* dphi, const double* dlnA, double* phi_out, double* dphi_out) {
  Mech* m = static_cast<Mech*>(h);
  const int N = m->K;
  const double p = p_Pa * 10.0;
  if (!dphi && !dlnA) {
    std::vector<double> y(phi, phi + N);
    for (int i = 0; i < n; ++i)
      if (!ros_step<double>(*m, p, y, hs[i], lnA_shift)) return 1;
    for (int i = 0; i < N; ++i) phi_out[i] = y[i];
    return 0;
  }
  std::vector<Dual> y(N), shift(m->R);
  for (int i = 0; i < N; ++i) y[i] = Dual(phi[i], dphi ? dphi[i] : 0.0);
  for (int r = 0; r < m->R; ++r) shift[r] = Dual(lnA_shift ? lnA_shift[r] : 0.0, dlnA ? dlnA[r] : 0.0);
  for (int i = 0; i < n; ++i)
    if (!ros_step<Dual>(*m, p, y, hs[i], shift.data())) return 1;
  for (int i = 0; i < N; ++i) { phi_out[i] = y[i].v; if (dphi_out) dphi_out[i] = y[i].d; }
  return 0;
}

// Rosenbrock coefficient table (classical form), for the order-condition tests:
// out = [gamma, alpha (16, row-major), gamma_ij (16), b (4), bhat (4)].
int oracle_ros_coefficients(double* out) {
  Ros4 c;
  out[0] = c.gamma;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) { out[1 + i * 4 + j] = c.alpha[i][j]; out[17 + i * 4 + j] = c.gam[i][j]; }
  for (int i = 0; i < 4; ++i) { out[33 + i] = c.b[i]; out[37 + i] = c.bhat[i]; }
  return 0;
}

// Algorithmic operation counts of one rate evaluation, one Jacobian evaluation, one LU factor
// and one LU solve at the given state.  counts[5 * 4] = {add, mul, div, exp, log} for
// [rates, jacobian (including its own rate evaluation), lu, solve].
int oracle_opcount(void* h, double p_Pa, double T, const double* Y, int64_t* counts) {
  Mech* m = static_cast<Mech*>(h);
  const int K = m->K, N = K;
  std::vector<Cnt> phi(N), fo(N), J((size_t)N * N);
  phi[0] = Cnt(T);
  for (int k = 0; k < K - 1; ++k) phi[1 + k] = Cnt(Y[k]);
  auto dump = [&](int slot) {
    counts[slot * 5 + 0] = g_ops.add; counts[slot * 5 + 1] = g_ops.mul; counts[slot * 5 + 2] = g_ops.div;
    counts[slot * 5 + 3] = g_ops.exp; counts[slot * 5 + 4] = g_ops.log;
    g_ops = OpCounts();
  };
  g_ops = OpCounts();
  {
    RateState<Cnt> st;
    rates(*m, p_Pa * 10.0, phi.data(), fo.data(), st);
  }
  dump(0);
  jacobian(*m, p_Pa * 10.0, phi.data(), fo.data(), J.data());
  dump(1);
  // LU and a solve on W = I/(gamma h) - J's pattern: use the identity-shifted Jacobian itself
  std::vector<Cnt> A(J);
  for (int i = 0; i < N; ++i) A[(size_t)i * N + i] = A[(size_t)i * N + i] + Cnt(1e6);
  g_ops = OpCounts();
  std::vector<int> piv(N);
  lu_factor(N, A.data(), piv.data());
  dump(2);
  std::vector<Cnt> b(N, Cnt(1.0));
  lu_solve(N, A.data(), piv.data(), b.data());
  dump(3);
  return 0;
}

}  // extern "C"
