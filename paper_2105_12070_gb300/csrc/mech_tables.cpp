// Mechanism file reader and device-table builder (host side of chem_load_mechanism).
//
// Two file formats: the generator's CHEMMECH text (see synth.py) and the common subset of
// CHEMKIN-II (ELEMENTS, SPECIES, THERMO with NASA-7 cards, REACTIONS).  Species carry NASA-7
// polynomials; reactions are reversible, with up to two reactant and two product molecules, of
// type elementary, third-body (+M), Lindemann or Troe fall-off ((+M) with LOW, TROE) (Sec. 2.3
// delegates these forms to the mechanism; the tables here only re-arrange them for the kernels).
#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <array>
#include <map>
#include <sstream>

#include "chem_internal.h"

namespace chemgpu {

namespace {

constexpr double kRcal = 8.314462618 / 4.184;  // cal/(mol K)

struct Reader {
  FILE* f = nullptr;
  char line[1 << 16];
  char* cur = nullptr;
  bool next_line() {
    while (std::fgets(line, sizeof(line), f)) {
      char* p = line;
      while (*p == ' ' || *p == '\t') ++p;
      if (*p == '#' || *p == '\n' || *p == '\r' || *p == 0) continue;
      cur = p;
      return true;
    }
    return false;
  }
  bool word(char* out, size_t n) {
    while (*cur == ' ' || *cur == '\t') ++cur;
    size_t i = 0;
    while (*cur && *cur != ' ' && *cur != '\t' && *cur != '\n' && *cur != '\r' && i + 1 < n) out[i++] = *cur++;
    out[i] = 0;
    return i > 0;
  }
  bool num(double& v) {
    char* end;
    v = std::strtod(cur, &end);
    if (end == cur) return false;
    cur = end;
    return true;
  }
  bool inum(int& v) {
    char* end;
    long x = std::strtol(cur, &end, 10);
    if (end == cur) return false;
    cur = end;
    v = (int)x;
    return true;
  }
};

struct FileReaction {
  int type = 0, reac[2] = {-1, -1}, prod[2] = {-1, -1};
  int collider = -1;  // CHEMKIN '(+NAME)': the one species that acts as the third body
  double A = 0, b = 0, Ea = 0, A0 = 0, b0 = 0, Ea0 = 0, troe[4] = {0, 0, 0, 0};
  std::vector<double> eff;
};

// Gather plan of the Jacobian's mass-action part and the row lists of its efficiency part, for
// the species rows k < K-1 (the enthalpy row follows from them, see the kernels).
// Per-reaction scratch layout (see the kernels): 8 rows of R values, scr[u * R + r] with u =
// 0..3 dq/dC at the distinct slot species, 4 phi, 5 sum_j dq/dC_j C_j, 6 dq/dT, 7 reaction
// enthalpy (rows, so that the threads of consecutive reactions touch consecutive words).
void build_jacobian_plan(HostMech& m) {
  const int K = m.K, d = K - 1;
  struct Contrib { int dst, src, src2; double coef; };
  std::vector<Contrib> cs;
  for (int r = 0; r < m.R; ++r) {
    const int* ii = &m.rxi[(size_t)r * kRxInts];
    for (int u = 0; u < 4; ++u) {
      const int col = ii[4 + u];
      if (col < 0) continue;
      for (int rs = 0; rs < 4; ++rs) {
        const int row = ii[8 + rs];
        if (row < 0) continue;
        cs.push_back({row * K + col, u * m.R + r, -1, (double)ii[12 + rs]});
      }
    }
  }
  std::stable_sort(cs.begin(), cs.end(), [](const Contrib& a, const Contrib& b) { return a.dst < b.dst; });
  // entries, then ordered by decreasing list length so that threads of a pass get similar work
  std::vector<std::pair<int, int>> ent;  // (begin, end) into cs
  for (size_t i = 0; i < cs.size();) {
    size_t j = i;
    while (j < cs.size() && cs[j].dst == cs[i].dst) ++j;
    ent.push_back({(int)i, (int)j});
    i = j;
  }
  std::stable_sort(ent.begin(), ent.end(),
                   [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
                     return (a.second - a.first) > (b.second - b.first);
                   });
  m.zg_ptr.assign(1, 0);
  m.zg_dst.clear(); m.zg_src.clear(); m.zg_src2.clear(); m.zg_coef.clear();
  for (const auto& e : ent) {
    m.zg_dst.push_back(cs[e.first].dst);
    for (int i = e.first; i < e.second; ++i) {
      m.zg_src.push_back(cs[i].src);
      m.zg_src2.push_back(cs[i].src2);
      m.zg_coef.push_back(cs[i].coef);
    }
    m.zg_ptr.push_back((int)m.zg_src.size());
  }
  // efficiency rows
  m.pr_ptr.assign(K + 1, 0);
  m.pr_pd.clear(); m.pr_nu.clear();
  const int npd = m.n_tb + m.n_fo;
  for (int k = 0; k < K; ++k) {
    m.pr_ptr[k] = (int)m.pr_pd.size();
    for (int p = 0; p < npd && k < d; ++p) {
      const int* ii = &m.rxi[(size_t)p * kRxInts];
      for (int rs = 0; rs < 4; ++rs)
        if (ii[8 + rs] == k) { m.pr_pd.push_back(p); m.pr_nu.push_back((double)ii[12 + rs]); }
    }
  }
  m.pr_ptr[K] = (int)m.pr_pd.size();
  m.pr_row.assign(m.pr_pd.size(), 0);
  m.pr_rows.clear();
  for (int k = 0; k < K; ++k) {
    for (int c = m.pr_ptr[k]; c < m.pr_ptr[k + 1]; ++c) m.pr_row[c] = k;
    if (m.pr_ptr[k + 1] > m.pr_ptr[k]) m.pr_rows.push_back(k);
  }
  std::stable_sort(m.pr_rows.begin(), m.pr_rows.end(), [&](int a, int b) {
    return (m.pr_ptr[a + 1] - m.pr_ptr[a]) < (m.pr_ptr[b + 1] - m.pr_ptr[b]);
  });
  // column lists for products with J^T: for each species column j, the scratch entries
  // dq/dC_j (u * R + r) of the reactions that have j among their distinct slot species
  m.cl_ptr.assign(K + 1, 0);
  m.cl_src.clear(); m.cl_rx.clear();
  for (int j = 0; j < K; ++j) {
    m.cl_ptr[j] = (int)m.cl_src.size();
    for (int r = 0; r < m.R; ++r) {
      const int* ii = &m.rxi[(size_t)r * kRxInts];
      for (int u = 0; u < 4; ++u)
        if (ii[4 + u] == j) { m.cl_src.push_back(u * m.R + r); m.cl_rx.push_back(r); }
    }
  }
  m.cl_ptr[K] = (int)m.cl_src.size();
}

}  // namespace

namespace {

// The generator's CHEMMECH format (the header already checked by the caller).
bool read_chemmech(const char* path, HostMech& m, std::vector<FileReaction>& rx, std::string& err) {
  Reader rd;
  rd.f = std::fopen(path, "r");
  if (!rd.f) { err = std::string("cannot open mechanism file ") + path; return false; }
  struct Closer { FILE* f; ~Closer() { std::fclose(f); } } closer{rd.f};
  char w[64];
  auto fail = [&](const char* what) { err = std::string("mechanism ") + path + ": " + what; return false; };
  if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "CHEMMECH")) return fail("missing CHEMMECH header");
  if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "elements") || !rd.inum(m.E) || m.E < 1)
    return fail("bad elements line");
  for (int e = 0; e < m.E; ++e)
    if (!rd.next_line()) return fail("short element list");
  if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "species") || !rd.inum(m.K) || m.K < 2)
    return fail("bad species line");
  const int K = m.K;
  m.sp.assign((size_t)K * kSpDoubles, 0.0);
  for (int k = 0; k < K; ++k) {
    double W, tlo, tmid, thi, a;
    if (!rd.next_line() || !rd.word(w, sizeof w) || !rd.num(W) || !rd.num(tlo) || !rd.num(tmid) || !rd.num(thi))
      return fail("bad species record");
    for (int e = 0; e < m.E; ++e) {
      int c;
      if (!rd.inum(c)) return fail("bad composition");
    }
    if (!(W > 0)) return fail("non-positive molar mass");
    double* s = &m.sp[(size_t)k * kSpDoubles];
    s[0] = W;
    s[1] = 1.0 / W;
    s[2] = tmid;
    for (int i = 0; i < 14; ++i) {
      if (!rd.num(a)) return fail("short NASA coefficients");
      s[3 + i] = a;
    }
  }
  int R;
  if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "reactions") || !rd.inum(R) || R < 0)
    return fail("bad reactions line");
  rx.assign(R, FileReaction());
  for (int r = 0; r < R; ++r) {
    FileReaction& x = rx[r];
    int nr, np;
    if (!rd.next_line() || !rd.inum(x.type) || !rd.inum(nr) || !rd.inum(x.reac[0]) || !rd.inum(x.reac[1]) ||
        !rd.inum(np) || !rd.inum(x.prod[0]) || !rd.inum(x.prod[1]) || !rd.num(x.A) || !rd.num(x.b) || !rd.num(x.Ea))
      return fail("bad reaction record");
    if (x.type < 0 || x.type > 3) return fail("unknown reaction type");
    for (int s = 0; s < 2; ++s)
      if (x.reac[s] < -1 || x.reac[s] >= K || x.prod[s] < -1 || x.prod[s] >= K) return fail("species index out of range");
    if ((x.reac[0] < 0 && x.reac[1] < 0) || (x.prod[0] < 0 && x.prod[1] < 0)) return fail("empty reaction side");
    // the kernels expect slot 0 of each side to be filled
    if (x.reac[0] < 0) std::swap(x.reac[0], x.reac[1]);
    if (x.prod[0] < 0) std::swap(x.prod[0], x.prod[1]);
    if (!(x.A > 0)) return fail("non-positive pre-exponential factor");
    if (x.type >= 1) {
      if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "eff")) return fail("missing eff line");
      x.eff.resize(K);
      for (int k = 0; k < K; ++k)
        if (!rd.num(x.eff[k])) return fail("short eff line");
    }
    if (x.type >= 2) {
      if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "low") || !rd.num(x.A0) || !rd.num(x.b0) ||
          !rd.num(x.Ea0))
        return fail("missing low line");
      if (!(x.A0 > 0)) return fail("non-positive low-pressure factor");
    }
    if (x.type == 3) {
      if (!rd.next_line() || !rd.word(w, sizeof w) || std::strcmp(w, "troe") || !rd.num(x.troe[0]) ||
          !rd.num(x.troe[1]) || !rd.num(x.troe[2]) || !rd.num(x.troe[3]))
        return fail("missing troe line");
    }
  }
  return true;
}

// Checks common to both readers, then the kernels' tables.
bool build_tables(const char* path, HostMech& m, std::vector<FileReaction>& rx, std::string& err) {
  auto fail = [&](const std::string& what) { err = std::string("mechanism ") + path + ": " + what; return false; };
  const int K = m.K, R = (int)rx.size();
  for (FileReaction& x : rx) {
    for (int s = 0; s < 2; ++s)
      if (x.reac[s] < -1 || x.reac[s] >= K || x.prod[s] < -1 || x.prod[s] >= K) return fail("species index out of range");
    if ((x.reac[0] < 0 && x.reac[1] < 0) || (x.prod[0] < 0 && x.prod[1] < 0)) return fail("empty reaction side");
    if (x.reac[0] < 0) std::swap(x.reac[0], x.reac[1]);
    if (x.prod[0] < 0) std::swap(x.prod[0], x.prod[1]);
    if (!(x.A > 0)) return fail("non-positive pre-exponential factor");
    if (x.type >= 1 && (int)x.eff.size() != K) return fail("missing collision efficiencies");
    if (x.type >= 2 && !(x.A0 > 0)) return fail("non-positive low-pressure factor");
  }
  // device order: Troe, Lindemann, third-body, elementary (stable within each kind): the
  // fall-off reactions, the costliest, fill whole 32-lane passes from index 0
  m.R = R;
  m.order.clear();
  for (int t = 3; t >= 0; --t)
    for (int r = 0; r < R; ++r)
      if (rx[r].type == t) m.order.push_back(r);
  m.n_elem = m.n_tb = m.n_fo = 0;
  for (int r = 0; r < R; ++r) {
    if (rx[r].type == kElementary) m.n_elem++;
    else if (rx[r].type == kThirdBody) m.n_tb++;
    else m.n_fo++;
  }
  m.rxd.assign((size_t)R * kRxDoubles, 0.0);
  m.rxi.assign((size_t)R * kRxInts, -1);
  m.dnu.assign(R, 0);
  m.eff.assign((size_t)(m.n_tb + m.n_fo) * K, 0.0);
  m.fo.assign((size_t)m.n_fo * kFoDoubles, 0.0);
  std::vector<std::vector<int>> sr(K);
  for (int dr = 0; dr < R; ++dr) {
    const FileReaction& x = rx[m.order[dr]];
    double* d = &m.rxd[(size_t)dr * kRxDoubles];
    d[0] = std::log(x.A);
    d[1] = x.b;
    d[2] = x.Ea / kRcal;
    int* ii = &m.rxi[(size_t)dr * kRxInts];
    ii[0] = x.reac[0]; ii[1] = x.reac[1]; ii[2] = x.prod[0]; ii[3] = x.prod[1];
    int nu_of[4] = {0, 0, 0, 0};
    int uc = 0;
    for (int s = 0; s < 4; ++s) {
      int sp = ii[s];
      if (sp < 0) continue;
      bool seen = false;
      for (int u = 0; u < uc; ++u) seen |= (ii[4 + u] == sp);
      if (!seen) ii[4 + uc++] = sp;
    }
    // net coefficients of the distinct slot species
    for (int u = 0; u < uc; ++u) {
      int sp = ii[4 + u], nu = 0;
      for (int s = 0; s < 2; ++s) {
        if (ii[s] == sp) nu -= 1;
        if (ii[2 + s] == sp) nu += 1;
      }
      nu_of[u] = nu;
      if (nu != 0) sr[sp].push_back(dr * 8 + (nu + 4));  // reaction and coefficient, unpacked below
    }
    int nrow = 0;
    for (int u = 0; u < uc; ++u)
      if (nu_of[u] != 0 && ii[4 + u] < K - 1) { ii[8 + nrow] = ii[4 + u]; ii[12 + nrow] = nu_of[u]; ++nrow; }
    for (int s = nrow; s < 4; ++s) ii[12 + s] = 0;
    for (int s = 0; s < 4; ++s) d[3 + s] = (double)ii[12 + s];
    m.dnu[dr] = (ii[2] >= 0) + (ii[3] >= 0) - (ii[0] >= 0) - (ii[1] >= 0);
    if (x.type >= 1) {
      const int pd = dr;  // pressure-dependent reactions come first
      for (int k = 0; k < K; ++k) m.eff[(size_t)pd * K + k] = x.eff[k];
    }
    if (x.type >= 2) {
      const int f = dr;  // fall-off reactions come first of all
      double* q = &m.fo[(size_t)f * kFoDoubles];
      q[0] = std::log(x.A0); q[1] = x.b0; q[2] = x.Ea0 / kRcal;
      q[3] = x.troe[0]; q[4] = x.troe[1]; q[5] = x.troe[2]; q[6] = x.troe[3];
      q[7] = (x.type == kTroe) ? 1.0 : 0.0;
      q[8] = (x.type == kTroe) ? 1.0 / x.troe[1] : 0.0;
      q[9] = (x.type == kTroe) ? 1.0 / x.troe[2] : 0.0;
    }
  }
  m.sr_ptr.assign(K + 1, 0);
  m.sr_idx.clear();
  m.sr_nu.clear();
  for (int k = 0; k < K; ++k) {
    m.sr_ptr[k] = (int)m.sr_idx.size();
    for (int code : sr[k]) {
      m.sr_idx.push_back(code >> 3);
      m.sr_nu.push_back((double)((code & 7) - 4));
    }
  }
  m.sr_ptr[K] = (int)m.sr_idx.size();
  build_jacobian_plan(m);
  return true;
}

// ------------------------------------------------------------------------------------------
// CHEMKIN-II reader (the common subset).
//   ELEMENTS: symbols, optionally with /atomic mass/ (default masses for H, C, O, N, AR, HE).
//   SPECIES: names.
//   THERMO [ALL]: optional line of default Tlow Tmid Thigh, then 80-column cards of four lines:
//     name (cols 1-18), four (element, count) pairs (cols 25-44), Tlow (46-55), Thigh (56-65),
//     Tmid (66-73, default if blank); then the 7 high-range and 7 low-range coefficients in
//     15-column fields, five per line.
//   REACTIONS [units]: "equation A b E" lines, equation sides joined by <=> or = (reversible);
//     '+M' makes a third-body reaction, '(+M)' a fall-off reaction (LOW / A0 b0 E0 / required,
//     TROE / alpha T3 T1 [T2] / optional: Troe, else Lindemann); efficiency lines NAME/value/;
//     DUPLICATE is accepted.  E units: CAL/MOLE (default), KCAL/MOLE, JOULES/MOLE, KJOULES/MOLE,
//     KELVINS; A in mol, cm, s.
//   Not supported (a clear error): irreversible '=>', explicit REV, PLOG, SRI, chemically
//   activated HIGH, more than two molecules on a side.  A named third body '(+AR)' makes the
//   collision efficiency 1 for that species and 0 for the others.

std::string upper(std::string s) {
  for (char& c : s) c = (char)std::toupper((unsigned char)c);
  return s;
}

std::string trim(const std::string& s) {
  size_t a = s.find_first_not_of(" \t\r\n"), b = s.find_last_not_of(" \t\r\n");
  return a == std::string::npos ? std::string() : s.substr(a, b - a + 1);
}

bool to_double(const std::string& t, double& v) {
  if (t.empty()) return false;
  char* end;
  std::string u = t;
  for (char& c : u) if (c == 'D' || c == 'd') c = 'E';  // Fortran exponents
  v = std::strtod(u.c_str(), &end);
  return end != u.c_str() && *end == 0;
}

bool read_chemkin(const char* path, HostMech& m, std::vector<FileReaction>& rx, std::string& err) {
  std::ifstream in(path);
  if (!in) { err = std::string("cannot open mechanism file ") + path; return false; }
  auto fail = [&](const std::string& what) { err = std::string("mechanism ") + path + ": " + what; return false; };
  std::vector<std::string> lines;
  for (std::string l; std::getline(in, l);) {
    const size_t c = l.find('!');
    if (c != std::string::npos) l = l.substr(0, c);
    if (!l.empty() && l.back() == '\r') l.pop_back();
    lines.push_back(l);
  }
  const std::map<std::string, double> default_mass = {{"H", 1.00797}, {"C", 12.01115}, {"O", 15.9994},
                                                      {"N", 14.0067}, {"AR", 39.948}, {"HE", 4.0026}};
  std::vector<std::string> el_names, sp_names;
  std::vector<double> el_mass;
  std::map<std::string, int> sp_index;
  size_t i = 0;
  auto first_word = [&](const std::string& l) {
    std::istringstream ss(l);
    std::string w;
    ss >> w;
    return upper(w);
  };
  // ELEMENTS and SPECIES (free format, may span lines; END closes a section)
  auto read_list = [&](std::vector<std::string>& toks) {
    std::istringstream ss(lines[i]);
    std::string w;
    ss >> w;  // the keyword
    for (;;) {
      while (ss >> w) {
        if (upper(w) == "END") return true;
        toks.push_back(w);
      }
      if (++i >= lines.size()) return false;
      ss.clear();
      ss.str(lines[i]);
      const std::string fw = first_word(lines[i]);
      if (fw.rfind("SPEC", 0) == 0 || fw.rfind("THER", 0) == 0 || fw.rfind("REAC", 0) == 0) {
        --i;
        return true;
      }
    }
  };
  bool have_thermo = false, have_reactions = false;
  std::vector<std::array<double, 17>> sp_data;
  std::vector<std::vector<int>> comp;
  for (; i < lines.size(); ++i) {
    const std::string fw = first_word(lines[i]);
    if (fw.empty()) continue;
    if (fw.rfind("ELEM", 0) == 0) {
      std::vector<std::string> toks;
      if (!read_list(toks)) return fail("unterminated ELEMENTS");
      // split "H/1.008/" and "H /1.008/" forms
      std::string joined;
      for (auto& t : toks) joined += t + " ";
      std::string name;
      for (size_t p = 0; p < joined.size();) {
        if (joined[p] == ' ') { ++p; continue; }
        if (joined[p] == '/') {
          const size_t q = joined.find('/', p + 1);
          if (q == std::string::npos || el_names.empty()) return fail("bad element mass");
          double v;
          if (!to_double(trim(joined.substr(p + 1, q - p - 1)), v) || !(v > 0)) return fail("bad element mass");
          el_mass.back() = v;
          p = q + 1;
          continue;
        }
        size_t q = p;
        while (q < joined.size() && joined[q] != ' ' && joined[q] != '/') ++q;
        name = upper(joined.substr(p, q - p));
        el_names.push_back(name);
        auto it = default_mass.find(name);
        el_mass.push_back(it == default_mass.end() ? -1.0 : it->second);
        p = q;
      }
    } else if (fw.rfind("SPEC", 0) == 0) {
      std::vector<std::string> toks;
      if (!read_list(toks)) return fail("unterminated SPECIES");
      for (auto& t : toks) {
        if (sp_index.count(upper(t))) return fail("duplicate species " + t);
        sp_index[upper(t)] = (int)sp_names.size();
        sp_names.push_back(t);
      }
    } else if (fw.rfind("THER", 0) == 0) {
      have_thermo = true;
      for (const std::string& e : el_names)
        if (el_mass[&e - &el_names[0]] <= 0) return fail("no atomic mass for element " + e);
      sp_data.assign(sp_names.size(), std::array<double, 17>());
      comp.assign(sp_names.size(), std::vector<int>(el_names.size(), 0));
      std::vector<bool> seen(sp_names.size(), false);
      double tdef[3] = {300.0, 1000.0, 5000.0};
      ++i;
      // optional line of default temperatures
      if (i < lines.size()) {
        std::istringstream ss(lines[i]);
        double a, b, c;
        if ((lines[i].size() < 80 || lines[i][79] != '1') && (ss >> a >> b >> c)) {
          tdef[0] = a; tdef[1] = b; tdef[2] = c;
          ++i;
        }
      }
      for (; i < lines.size(); ++i) {
        const std::string& l = lines[i];
        if (first_word(l) == "END") break;
        if (trim(l).empty()) continue;
        if (l.size() < 80 || l[79] != '1') continue;  // not the first line of a card
        if (i + 3 >= lines.size()) return fail("truncated thermo card");
        const std::string name = upper(trim(l.substr(0, 18)).substr(0, trim(l.substr(0, 18)).find(' ')));
        auto it = sp_index.find(name);
        if (it == sp_index.end()) { i += 3; continue; }  // a species this mechanism does not use
        const int k = it->second;
        for (int e = 0; e < 4; ++e) {
          const std::string sym = upper(trim(l.substr(24 + 5 * e, 2)));
          const std::string cnt = trim(l.substr(26 + 5 * e, 3));
          if (sym.empty() || sym == "0") continue;
          double c;
          if (!to_double(cnt, c)) return fail("bad element count for " + name);
          auto pos = std::find(el_names.begin(), el_names.end(), sym);
          if (pos == el_names.end()) {
            if (c != 0) return fail("undeclared element " + sym + " in " + name);
            continue;
          }
          comp[k][pos - el_names.begin()] += (int)std::lround(c);
        }
        double tlo, thi, tmid;
        if (!to_double(trim(l.substr(45, 10)), tlo)) tlo = tdef[0];
        if (!to_double(trim(l.substr(55, 10)), thi)) thi = tdef[2];
        if (!to_double(trim(l.size() >= 73 ? l.substr(65, 8) : std::string()), tmid)) tmid = tdef[1];
        (void)tlo;
        (void)thi;
        double a[15];
        int na = 0;
        for (int r = 1; r <= 3; ++r) {
          const std::string& cl = lines[i + r];
          for (int f = 0; f < 5 && na < 14; ++f) {
            if ((int)cl.size() < 15 * (f + 1)) return fail("short thermo card for " + name);
            if (!to_double(trim(cl.substr(15 * f, 15)), a[na])) return fail("bad thermo coefficient for " + name);
            ++na;
          }
        }
        std::array<double, 17>& s = sp_data[k];
        s[2] = tmid;
        for (int q = 0; q < 7; ++q) { s[3 + q] = a[7 + q]; s[10 + q] = a[q]; }  // low range, then high
        seen[k] = true;
        i += 3;
      }
      for (size_t k = 0; k < sp_names.size(); ++k)
        if (!seen[k]) return fail("no thermo data for species " + sp_names[k]);
    } else if (fw.rfind("REAC", 0) == 0) {
      have_reactions = true;
      double e_scale = 1.0;  // to cal/mol
      {
        std::istringstream ss(lines[i]);
        std::string w;
        ss >> w;
        while (ss >> w) {
          const std::string u = upper(w);
          if (u == "CAL/MOLE") e_scale = 1.0;
          else if (u == "KCAL/MOLE") e_scale = 1000.0;
          else if (u == "JOULES/MOLE") e_scale = 1.0 / 4.184;
          else if (u == "KJOULES/MOLE") e_scale = 1000.0 / 4.184;
          else if (u == "KELVINS") e_scale = kRcal;
          else if (u == "MOLES") {}
          else return fail("unsupported REACTIONS unit " + w);
        }
      }
      const int K = (int)sp_names.size();
      for (++i; i < lines.size(); ++i) {
        const std::string l = trim(lines[i]);
        if (l.empty()) continue;
        if (first_word(l) == "END") break;
        if (l.find('=') != std::string::npos) {
          // equation A b E: the last three tokens are numbers, the rest is the equation
          std::istringstream ss(l);
          std::vector<std::string> t;
          for (std::string w; ss >> w;) t.push_back(w);
          if (t.size() < 4) return fail("bad reaction line: " + l);
          FileReaction x;
          if (!to_double(t[t.size() - 3], x.A) || !to_double(t[t.size() - 2], x.b) ||
              !to_double(t[t.size() - 1], x.Ea))
            return fail("bad Arrhenius parameters: " + l);
          x.Ea *= e_scale;
          std::string eq;
          for (size_t q = 0; q + 3 < t.size(); ++q) eq += t[q];
          std::string ueq = upper(eq);
          size_t sep;
          size_t seplen;
          if ((sep = ueq.find("<=>")) != std::string::npos) seplen = 3;
          else if (ueq.find("=>") != std::string::npos) return fail("irreversible reaction not supported: " + eq);
          else if ((sep = ueq.find('=')) != std::string::npos) seplen = 1;
          else return fail("no '=' in reaction: " + eq);
          std::string side[2] = {ueq.substr(0, sep), ueq.substr(sep + seplen)};
          bool falloff[2] = {false, false}, third[2] = {false, false};
          int collider[2] = {-1, -1};
          std::vector<int> mol[2];
          for (int sd = 0; sd < 2; ++sd) {
            std::string& sv = side[sd];
            const size_t fp = sv.find("(+");
            if (fp != std::string::npos) {
              // '(+M)', or '(+NAME)': that species alone is the third body of the fall-off
              const std::string c = sv.substr(fp + 2);
              if (c.size() < 2 || c.back() != ')') return fail("bad third body in " + eq);
              const std::string name = c.substr(0, c.size() - 1);
              if (name != "M") {
                auto it = sp_index.find(name);
                if (it == sp_index.end()) return fail("unknown third body " + name + " in " + eq);
                collider[sd] = it->second;
              }
              falloff[sd] = true;
              sv = sv.substr(0, fp);
            }
            std::vector<std::string> terms;
            size_t a = 0;
            for (size_t p = 0; p <= sv.size(); ++p)
              if (p == sv.size() || sv[p] == '+') { terms.push_back(sv.substr(a, p - a)); a = p + 1; }
            for (const std::string& term : terms) {
              if (term.empty()) return fail("empty term in " + eq);
              if (term == "M") { third[sd] = true; continue; }
              size_t d = 0;
              while (d < term.size() && std::isdigit((unsigned char)term[d])) ++d;
              const int coef = d ? std::atoi(term.substr(0, d).c_str()) : 1;
              auto it = sp_index.find(term.substr(d));
              if (it == sp_index.end()) return fail("unknown species " + term.substr(d) + " in " + eq);
              for (int c = 0; c < coef; ++c) mol[sd].push_back(it->second);
            }
          }
          if (falloff[0] != falloff[1] || third[0] != third[1]) return fail("unbalanced +M in " + eq);
          if (falloff[0] && third[0]) return fail("both +M and (+M) in " + eq);
          if (collider[0] != collider[1]) return fail("different third bodies on the two sides of " + eq);
          for (int sd = 0; sd < 2; ++sd)
            if (mol[sd].empty() || mol[sd].size() > 2) return fail("one or two molecules per side only: " + eq);
          x.reac[0] = mol[0][0]; x.reac[1] = mol[0].size() > 1 ? mol[0][1] : -1;
          x.prod[0] = mol[1][0]; x.prod[1] = mol[1].size() > 1 ? mol[1][1] : -1;
          x.type = falloff[0] ? kLindemann : (third[0] ? kThirdBody : kElementary);
          x.collider = collider[0];
          if (x.type >= kThirdBody) x.eff.assign(K, x.collider >= 0 ? 0.0 : 1.0);
          if (x.collider >= 0) x.eff[x.collider] = 1.0;
          rx.push_back(x);
          continue;
        }
        // auxiliary lines of the last reaction
        if (rx.empty()) return fail("auxiliary line before any reaction: " + l);
        FileReaction& x = rx.back();
        const std::string ul = upper(l);
        auto slash_values = [&](const std::string& key, std::vector<double>& v) {
          const size_t a = ul.find('/'), b = ul.rfind('/');
          if (a == std::string::npos || b == a) return false;
          std::istringstream ss(l.substr(a + 1, b - a - 1));
          for (std::string w; ss >> w;) {
            double d;
            if (!to_double(w, d)) return false;
            v.push_back(d);
          }
          (void)key;
          return true;
        };
        const std::string kw = ul.substr(0, ul.find_first_of(" /"));
        if (kw == "DUP" || kw == "DUPLICATE") continue;
        if (kw == "LOW") {
          std::vector<double> v;
          if (x.type != kLindemann && x.type != kTroe) return fail("LOW without (+M): " + l);
          if (!slash_values(kw, v) || v.size() != 3) return fail("bad LOW: " + l);
          x.A0 = v[0]; x.b0 = v[1]; x.Ea0 = v[2] * e_scale;
          continue;
        }
        if (kw == "TROE") {
          std::vector<double> v;
          if (x.type != kLindemann && x.type != kTroe) return fail("TROE without (+M): " + l);
          if (!slash_values(kw, v) || (v.size() != 3 && v.size() != 4)) return fail("bad TROE: " + l);
          x.type = kTroe;
          x.troe[0] = v[0]; x.troe[1] = v[1]; x.troe[2] = v[2];
          x.troe[3] = v.size() == 4 ? v[3] : 1e30;  // no third term: exp(-T2/T) = 0
          continue;
        }
        if (kw == "REV" || kw == "PLOG" || kw == "SRI" || kw == "HIGH" || kw == "FORD" || kw == "RORD" ||
            kw == "CHEB" || kw == "UNITS" || kw == "LT" || kw == "RLT" || kw == "TDEP" || kw == "EXCI")
          return fail("unsupported reaction keyword " + kw);
        // efficiencies: NAME/value/ NAME/value/ ...
        if (x.type == kElementary) return fail("efficiencies for a reaction without +M: " + l);
        if (x.collider >= 0) return fail("efficiencies for a reaction with a named third body: " + l);
        size_t p = 0;
        while (p < l.size()) {
          while (p < l.size() && (l[p] == ' ' || l[p] == '\t')) ++p;
          if (p >= l.size()) break;
          const size_t a = l.find('/', p);
          const size_t b = a == std::string::npos ? a : l.find('/', a + 1);
          if (b == std::string::npos) return fail("bad efficiency list: " + l);
          const std::string nm = upper(trim(l.substr(p, a - p)));
          double v;
          if (!to_double(trim(l.substr(a + 1, b - a - 1)), v)) return fail("bad efficiency: " + l);
          auto it = sp_index.find(nm);
          if (it == sp_index.end()) return fail("unknown species in efficiencies: " + nm);
          x.eff[it->second] = v;
          p = b + 1;
        }
      }
    }
  }
  if (sp_names.size() < 2 || !have_thermo || !have_reactions) return fail("need SPECIES, THERMO and REACTIONS");
  for (const FileReaction& x : rx)
    if ((x.type == kLindemann || x.type == kTroe) && !(x.A0 > 0)) return fail("fall-off reaction without LOW");
  m.E = (int)el_names.size();
  m.K = (int)sp_names.size();
  m.sp.assign((size_t)m.K * kSpDoubles, 0.0);
  for (int k = 0; k < m.K; ++k) {
    double W = 0.0;
    for (int e = 0; e < m.E; ++e) W += comp[k][e] * el_mass[e];
    if (!(W > 0)) return fail("species " + sp_names[k] + " has no mass");
    double* s = &m.sp[(size_t)k * kSpDoubles];
    s[0] = W;
    s[1] = 1.0 / W;
    for (int q = 2; q < 17; ++q) s[q] = sp_data[k][q];
  }
  return true;
}

}  // namespace

bool parse_mechanism(const char* path, HostMech& m, std::string& err) {
  // CHEMMECH files start with that word; anything else is read as CHEMKIN-II
  bool chemmech = false;
  {
    std::ifstream in(path);
    if (!in) { err = std::string("cannot open mechanism file ") + path; return false; }
    for (std::string l; std::getline(in, l);) {
      const std::string t = trim(l);
      if (t.empty() || t[0] == '#' || t[0] == '!') continue;
      chemmech = t.rfind("CHEMMECH", 0) == 0;
      break;
    }
  }
  std::vector<FileReaction> rx;
  if (!(chemmech ? read_chemmech(path, m, rx, err) : read_chemkin(path, m, rx, err))) return false;
  return build_tables(path, m, rx, err);
}

}  // namespace chemgpu
