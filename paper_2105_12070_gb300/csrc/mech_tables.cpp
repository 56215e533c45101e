// Mechanism file reader and device-table builder (host side of chem_load_mechanism).
//
// File format: see the generator (synth.py).  Species carry molar mass and NASA-7
// polynomials; reactions are reversible, with up to two reactants and two products, of type
// elementary, third-body, Lindemann or Troe fall-off (Sec. 2.3 delegates these forms to the
// mechanism; the tables here only re-arrange them for the kernels).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

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

bool parse_mechanism(const char* path, HostMech& m, std::string& err) {
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
  std::vector<FileReaction> rx(R);
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

}  // namespace chemgpu
