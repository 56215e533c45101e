"""Seeded synthetic inputs: reaction mechanisms and cell fields.

This module only draws inputs.  It holds none of the chemistry-solve arithmetic
(no rates, no Jacobian, no integrator): it produces a mechanism file and arrays
of initial states that both the CUDA library and the CPU oracle read, each with
its own code.

The paper's cases use real mechanisms (GRI-3.0 with 53 species / 325 reactions,
Sec. 2.3; Yao with 54 / 269, Sec. 3.2; DRM19 with 21 / 83, Sec. 3.5) that are
not available here.  The mechanisms below are synthetic stand-ins of the same
sizes and reaction-type mix, drawn from a seed:

* species: distinct non-zero integer element compositions (0-3 atoms of each
  element); molar mass from the element masses;
* thermo: NASA 7-coefficient polynomials (two ranges split at 1000 K) fitted by
  least squares to a smooth model heat capacity
  cp/R = c0 + (cinf - c0)(1 - exp(-T/theta)), c0 = 3.5,
  cinf = 3.5 + 1.5 (atoms - 1), theta ~ U[500, 1500] K, with cp continuous at
  1000 K; the enthalpy and entropy constants come from
  h_f(298.15 K) = 50 atoms - 80 (atoms - 1) + U[-25, 25] kcal/mol (an atom
  term minus one bond energy per extra atom) and
  s(298.15 K) = 35 + 4.5 atoms + U[-3, 3] cal/(mol K), and the high-range
  constants make h and s continuous at 1000 K.  With independent uniform h_f
  and s (no bond structure) one direction of most reactions gets a reverse
  rate constant 1e10-1e30 above collision rates, which no real mechanism has;
* reactions: element-balanced, reversible, from the templates A+B=C+D, A+B=C
  and A=B+C (equal odds), found by hashing sums of composition vectors; each
  reaction is written in its exothermic direction (298 K formation
  enthalpies), as real mechanisms quote the Arrhenius fit of that direction,
  so that reverse rates k_f/Kc carry a positive activation energy;
  log10 A ~ U[8, 14] (cgs), b ~ U[-1, 2], Ea ~ U[0, 50] kcal/mol;
  third-body and fall-off reactions use the A+B=C / A=B+C templates, with
  collision efficiencies ~ U[0.5, 5] for every species; fall-off low-pressure
  limits log10 A0 ~ U[14, 18], b0 ~ U[-2, 0], E0 ~ U[0, 30] kcal/mol; Troe
  parameters alpha ~ U[0.1, 0.9], T3 ~ U[50, 500], T1 ~ U[500, 5000],
  T2 ~ U[2000, 8000] K.

Mechanism file format (text, one record per line, '#' starts a comment line)::

    CHEMMECH 1
    elements E
    <name> <atomic mass g/mol>                                  (E lines)
    species K
    <name> <W g/mol> <Tlow> <Tmid> <Thigh> <E composition ints> <7 low coeffs> <7 high coeffs>
    reactions R
    <type> <nr> <r1> <r2> <np> <p1> <p2> <A> <b> <Ea cal/mol>
    eff <K efficiencies>                    (types 1, 2, 3)
    low <A0> <b0> <Ea0 cal/mol>             (types 2, 3)
    troe <alpha> <T3> <T1> <T2>             (type 3)
    end

Reaction types: 0 elementary, 1 third body (+M), 2 Lindemann fall-off,
3 Troe fall-off.  Species indices are 0-based, -1 marks an unused slot.  A is in
mol, cm, s units for the forward reaction as written (a third-body A includes
the [M] order).  Floats are written with 17 significant digits so that a reader
using strtod recovers the same doubles.
"""
from __future__ import annotations

import os
import tempfile
from dataclasses import dataclass, field

import numpy as np

ELEMENT_MASS = {"H": 1.008, "C": 12.011, "O": 15.999, "N": 14.007}
ELEMENT_ORDER = ["H", "C", "O", "N"]
P_ATM_PA = 101325.0

T_LOW, T_MID, T_HIGH, T_REF = 300.0, 1000.0, 5000.0, 298.15
R_CAL = 1.98720425864083  # cal/(mol K), only used to turn h_f, s_298 draws into NASA constants

TYPE_ELEMENTARY, TYPE_THIRD_BODY, TYPE_LINDEMANN, TYPE_TROE = 0, 1, 2, 3


@dataclass
class Mechanism:
    seed: int
    elements: list
    element_mass: np.ndarray  # [E]
    comp: np.ndarray  # [K, E] int
    W: np.ndarray  # [K]
    a_low: np.ndarray  # [K, 7]
    a_high: np.ndarray  # [K, 7]
    rtype: np.ndarray  # [R] int
    reac: np.ndarray  # [R, 2] int, -1 unused
    prod: np.ndarray  # [R, 2] int, -1 unused
    A: np.ndarray  # [R]
    b: np.ndarray  # [R]
    Ea: np.ndarray  # [R] cal/mol
    eff: dict = field(default_factory=dict)  # r -> [K]
    low: dict = field(default_factory=dict)  # r -> (A0, b0, Ea0)
    troe: dict = field(default_factory=dict)  # r -> (alpha, T3, T1, T2)

    @property
    def K(self) -> int:
        return self.comp.shape[0]

    @property
    def R(self) -> int:
        return self.rtype.shape[0]

    def species_names(self):
        return [f"S{k}" for k in range(self.K)]

    def write(self, path: str) -> str:
        f17 = lambda x: repr(float(x))
        lines = ["CHEMMECH 1", f"# synthetic mechanism, seed {self.seed}"]
        lines.append(f"elements {len(self.elements)}")
        for e, m in zip(self.elements, self.element_mass):
            lines.append(f"{e} {f17(m)}")
        lines.append(f"species {self.K}")
        for k in range(self.K):
            toks = [f"S{k}", f17(self.W[k]), f17(T_LOW), f17(T_MID), f17(T_HIGH)]
            toks += [str(int(c)) for c in self.comp[k]]
            toks += [f17(a) for a in self.a_low[k]] + [f17(a) for a in self.a_high[k]]
            lines.append(" ".join(toks))
        lines.append(f"reactions {self.R}")
        for r in range(self.R):
            nr = int((self.reac[r] >= 0).sum())
            npr = int((self.prod[r] >= 0).sum())
            toks = [str(int(self.rtype[r])), str(nr), str(int(self.reac[r, 0])), str(int(self.reac[r, 1])),
                    str(npr), str(int(self.prod[r, 0])), str(int(self.prod[r, 1])),
                    f17(self.A[r]), f17(self.b[r]), f17(self.Ea[r])]
            lines.append(" ".join(toks))
            if self.rtype[r] >= TYPE_THIRD_BODY:
                lines.append("eff " + " ".join(f17(x) for x in self.eff[r]))
            if self.rtype[r] >= TYPE_LINDEMANN:
                lines.append("low " + " ".join(f17(x) for x in self.low[r]))
            if self.rtype[r] == TYPE_TROE:
                lines.append("troe " + " ".join(f17(x) for x in self.troe[r]))
        lines.append("end")
        with open(path, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        return path

    def rounded(self, digits: int = 9):
        """A copy whose NASA coefficients carry `digits` significant digits (what the E15.8 fields of
        a CHEMKIN thermo card hold), so that its CHEMMECH and CHEMKIN files describe the same
        numbers."""
        import copy
        m = copy.deepcopy(self)
        r = lambda a: np.array([float(f"{x:.{digits - 1}e}") for x in np.ravel(a)]).reshape(np.shape(a))
        m.a_low, m.a_high = r(self.a_low), r(self.a_high)
        m.W = self.comp @ self.element_mass
        return m

    def write_chemkin(self, path: str) -> str:
        """The mechanism in CHEMKIN-II text: ELEMENTS (with their masses), SPECIES, THERMO (NASA-7
        cards, four 80-column lines per species, E15.8 coefficient fields) and REACTIONS (CAL/MOLE,
        MOLES; reversible '<=>', '+M' third bodies with efficiencies, '(+M)' fall-off with LOW and
        TROE)."""
        names = self.species_names()
        f17 = lambda x: repr(float(x))
        L = ["! synthetic mechanism, seed %d (CHEMKIN-II form)" % self.seed]
        L.append("ELEMENTS " + " ".join(f"{e} /{f17(mm)}/" for e, mm in zip(self.elements, self.element_mass)))
        L.append("END")
        L.append("SPECIES")
        for i in range(0, self.K, 8):
            L.append(" ".join(names[i:i + 8]))
        L.append("END")
        L.append("THERMO ALL")
        L.append(f"{T_LOW:10.3f}{T_MID:10.3f}{T_HIGH:10.3f}")
        for k in range(self.K):
            el = ""
            for e, c in zip(self.elements, self.comp[k]):
                el += f"{e:<2s}{int(c):3d}"
            el = el.ljust(20)[:20]
            head = f"{names[k]:<18s}{'SYN':6s}{el}G{T_LOW:10.3f}{T_HIGH:10.3f}{T_MID:8.2f}"
            L.append(head.ljust(79) + "1")
            co = list(self.a_high[k]) + list(self.a_low[k])
            fmt = lambda x: f"{x:15.8E}"
            L.append("".join(fmt(x) for x in co[0:5]).ljust(79) + "2")
            L.append("".join(fmt(x) for x in co[5:10]).ljust(79) + "3")
            L.append("".join(fmt(x) for x in co[10:14]).ljust(79) + "4")
        L.append("END")
        L.append("REACTIONS CAL/MOLE MOLES")
        for r in range(self.R):
            t = int(self.rtype[r])
            lhs = [names[i] for i in self.reac[r] if i >= 0]
            rhs = [names[i] for i in self.prod[r] if i >= 0]
            if t == TYPE_THIRD_BODY:
                lhs.append("M")
                rhs.append("M")
            eq = "+".join(lhs) + ("(+M)" if t >= TYPE_LINDEMANN else "") + "<=>" + "+".join(rhs) + \
                ("(+M)" if t >= TYPE_LINDEMANN else "")
            L.append(f"{eq:<40s} {f17(self.A[r])} {f17(self.b[r])} {f17(self.Ea[r])}")
            if t >= TYPE_LINDEMANN:
                L.append("    LOW / " + " ".join(f17(x) for x in self.low[r]) + " /")
            if t == TYPE_TROE:
                L.append("    TROE / " + " ".join(f17(x) for x in self.troe[r]) + " /")
            if t >= TYPE_THIRD_BODY:
                eff = self.eff[r]
                for i in range(0, self.K, 6):
                    L.append("    " + " ".join(f"{names[k]}/{f17(eff[k])}/" for k in range(i, min(self.K, i + 6))))
        L.append("END")
        with open(path, "w") as fh:
            fh.write("\n".join(L) + "\n")
        return path

    def write_temp(self) -> str:
        fd, path = tempfile.mkstemp(prefix=f"mech_s{self.seed}_", suffix=".txt")
        os.close(fd)
        return self.write(path)


# ----------------------------------------------------------------------------------------------
# thermo fit (input construction only)


def _fit_nasa7(rng, atoms: int):
    c0 = 3.5
    cinf = 3.5 + 1.5 * (atoms - 1)
    theta = rng.uniform(500.0, 1500.0)
    model = lambda T: c0 + (cinf - c0) * (1.0 - np.exp(-T / theta))
    # low range: degree-4 least squares in x = T/1000
    Tl = np.linspace(T_LOW, T_MID, 141)
    xl = Tl / 1000.0
    Vl = np.vander(xl, 5, increasing=True)
    cl = np.linalg.lstsq(Vl, model(Tl), rcond=None)[0]
    # high range: q(x) = p_low(1) + (x - 1) * cubic(x), so cp is continuous at 1000 K
    Th = np.linspace(T_MID, T_HIGH, 401)
    xh = Th / 1000.0
    p1 = cl.sum()
    Vh = np.vander(xh, 4, increasing=True) * (xh - 1.0)[:, None]
    r = np.linalg.lstsq(Vh, model(Th) - p1, rcond=None)[0]
    # expand p1 + (x-1)(r0 + r1 x + r2 x^2 + r3 x^3) into monomials of x
    ch = np.zeros(5)
    ch[0] = p1 - r[0]
    ch[1] = r[0] - r[1]
    ch[2] = r[1] - r[2]
    ch[3] = r[2] - r[3]
    ch[4] = r[3]
    scale = 1000.0 ** np.arange(5)
    return cl / scale, ch / scale  # coefficients of T^k


def _h_over_r_poly(a5, T):
    # integral of sum a_k T^k dT (without constant), i.e. enthalpy/R up to a constant
    return sum(a5[k] * T ** (k + 1) / (k + 1) for k in range(5))


def _s_over_r_poly(a5, T):
    # integral of sum a_k T^(k-1) dT (without constant), i.e. entropy/R up to a constant
    return a5[0] * np.log(T) + sum(a5[k] * T ** k / k for k in range(1, 5))


def _draw_thermo(rng, comp):
    K = comp.shape[0]
    a_low = np.zeros((K, 7))
    a_high = np.zeros((K, 7))
    h_f = np.zeros(K)
    for k in range(K):
        atoms = int(comp[k].sum())
        lo, hi = _fit_nasa7(rng, atoms)
        # formation enthalpy: atoms minus bonds (atoms - 1) plus noise, so that associations
        # release a bond energy (~80 kcal/mol) and exchanges are near-thermoneutral (+-50)
        hf = (50.0 * atoms - 80.0 * (atoms - 1) + rng.uniform(-25.0, 25.0)) * 1000.0  # cal/mol
        # standard entropy grows with size; associations then lose ~35 cal/(mol K)
        s0 = 35.0 + 4.5 * atoms + rng.uniform(-3.0, 3.0)  # cal/(mol K)
        a6l = hf / R_CAL - _h_over_r_poly(lo, T_REF)
        a7l = s0 / R_CAL - _s_over_r_poly(lo, T_REF)
        a6h = _h_over_r_poly(lo, T_MID) + a6l - _h_over_r_poly(hi, T_MID)
        a7h = _s_over_r_poly(lo, T_MID) + a7l - _s_over_r_poly(hi, T_MID)
        a_low[k, :5], a_low[k, 5], a_low[k, 6] = lo, a6l, a7l
        a_high[k, :5], a_high[k, 5], a_high[k, 6] = hi, a6h, a7h
        h_f[k] = hf
    return a_low, a_high, h_f


# ----------------------------------------------------------------------------------------------
# reactions


def _draw_species(rng, K, E):
    """Distinct non-zero compositions with 0-3 atoms per element.  Starting from the E one-atom
    species, most new species are the sum of two existing ones (as radicals combine in real
    mechanisms), which makes element-balanced reactions plentiful; the rest are uniform draws."""
    seen = set()
    comps = []

    def add(c):
        c = tuple(int(x) for x in c)
        if sum(c) == 0 or c in seen or max(c) > 3:
            return
        seen.add(c)
        comps.append(c)

    for e in range(min(E, K)):
        add(np.eye(E, dtype=np.int64)[e])
    while len(comps) < K:
        if rng.random() < 0.95:
            w = 1.0 / np.array([sum(c) for c in comps], dtype=float)
            a, b = rng.choice(len(comps), size=2, p=w / w.sum())
            add(np.array(comps[a]) + np.array(comps[b]))
        else:
            add(rng.integers(0, 4, size=E))
    return np.array(comps, dtype=np.int64)


def _candidates(comp):
    """All distinct balanced reactions: exchange pairs {A+B, C+D} and associations (A, B, C) with
    comp[A] + comp[B] == comp[C]."""
    K = comp.shape[0]
    index = {tuple(c): k for k, c in enumerate(comp)}
    by_sum = {}
    for a in range(K):
        for b in range(a, K):
            by_sum.setdefault(tuple(comp[a] + comp[b]), []).append((a, b))
    exchange = []
    combine = []
    for s, pairs in by_sum.items():
        for i in range(len(pairs)):
            for j in range(i + 1, len(pairs)):
                exchange.append((pairs[i], pairs[j]))
        if s in index:
            for (a, b) in pairs:
                combine.append(((a, b), (index[s],)))
    return exchange, combine


def make_mechanism(seed: int, K: int, R: int, n_elements: int = 3, n_third_body: int = 0,
                   n_lindemann: int = 0, n_troe: int = 0) -> Mechanism:
    """Draw a reversible, element-balanced mechanism with K species and R reactions.

    The first n_third_body + n_lindemann + n_troe reactions are the pressure-dependent ones
    (in that order); all use the association / dissociation templates.
    """
    rng = np.random.default_rng(seed)
    elements = ELEMENT_ORDER[:n_elements]
    emass = np.array([ELEMENT_MASS[e] for e in elements])
    n_pd = n_third_body + n_lindemann + n_troe
    for _attempt in range(100000):
        comp = _draw_species(rng, K, n_elements)
        exchange, combine = _candidates(comp)
        if len(exchange) + len(combine) >= R + 2 and len(combine) >= n_pd + 1:
            break
    else:  # pragma: no cover - the draws above always find enough candidates for the named sizes
        raise RuntimeError("could not draw a species set with enough balanced reactions")
    W = comp @ emass
    a_low, a_high, h_f = _draw_thermo(rng, comp)

    reac = np.full((R, 2), -1, dtype=np.int64)
    prod = np.full((R, 2), -1, dtype=np.int64)
    rtype = np.zeros(R, dtype=np.int64)
    pool = {0: [exchange[i] for i in rng.permutation(len(exchange))],
            1: [combine[i] for i in rng.permutation(len(combine))]}
    for r in range(R):
        # template: 0 = A+B=C+D, 1 = A+B=C, 2 = A=B+C (pressure-dependent reactions: 1 or 2)
        template = int(rng.integers(1, 3)) if r < n_pd else int(rng.integers(0, 3))
        kind = 0 if template == 0 else 1
        if not pool[kind]:
            kind = 1 - kind
            template = 0 if kind == 0 else 1
        lhs, rhs = pool[kind].pop()
        if sum(h_f[k] for k in rhs) > sum(h_f[k] for k in lhs):
            # written in the exothermic direction (298 K formation enthalpies), as mechanisms
            # quote the Arrhenius fit of that direction: the reverse rate k_f/Kc then carries a
            # positive activation energy.  The template fixes the shape of the reversible
            # reaction (A+B=C and A=B+C are its two directions).
            lhs, rhs = rhs, lhs
        reac[r, :len(lhs)] = lhs
        prod[r, :len(rhs)] = rhs
        if r < n_third_body:
            rtype[r] = TYPE_THIRD_BODY
        elif r < n_third_body + n_lindemann:
            rtype[r] = TYPE_LINDEMANN
        elif r < n_pd:
            rtype[r] = TYPE_TROE
    A = 10.0 ** rng.uniform(8.0, 14.0, size=R)
    b = rng.uniform(-1.0, 2.0, size=R)
    Ea = rng.uniform(0.0, 50.0, size=R) * 1000.0
    mech = Mechanism(seed, elements, emass, comp, W, a_low, a_high, rtype, reac, prod, A, b, Ea)
    for r in range(n_pd):
        mech.eff[r] = rng.uniform(0.5, 5.0, size=K)
        if rtype[r] >= TYPE_LINDEMANN:
            mech.low[r] = (10.0 ** rng.uniform(14.0, 18.0), rng.uniform(-2.0, 0.0), rng.uniform(0.0, 30.0) * 1000.0)
        if rtype[r] == TYPE_TROE:
            mech.troe[r] = (rng.uniform(0.1, 0.9), rng.uniform(50.0, 500.0), rng.uniform(500.0, 5000.0),
                            rng.uniform(2000.0, 8000.0))
    return mech


# ----------------------------------------------------------------------------------------------
# named mechanisms and cell fields


def mechanism_small() -> Mechanism:
    """10 species / 30 reactions / 3 elements, 3 third-body + 1 Lindemann (seed 1)."""
    return make_mechanism(1, 10, 30, n_elements=3, n_third_body=3, n_lindemann=1)


def mechanism_53() -> Mechanism:
    """53 species / 325 reactions / 4 elements, 30 third-body + 25 Troe (seed 2): GRI-3.0-sized."""
    return make_mechanism(2, 53, 325, n_elements=4, n_third_body=30, n_troe=25)


def mechanism_100() -> Mechanism:
    """100 species / 700 reactions / 4 elements, 60 third-body + 40 Troe (seed 3)."""
    return make_mechanism(3, 100, 700, n_elements=4, n_third_body=60, n_troe=40)


def cells_uniform(seed: int, K: int, n: int, T_range=(1000.0, 1800.0)):
    """n cells with T ~ U[T_range] and Y ~ Dirichlet(1); Y returned species-major [K, n]."""
    rng = np.random.default_rng(seed)
    T = rng.uniform(T_range[0], T_range[1], size=n)
    Y = rng.dirichlet(np.ones(K), size=n).T.copy()
    return T, Y


def _shear_streams(rng, K):
    return rng.dirichlet(np.ones(K)), rng.dirichlet(np.ones(K))


def shear_layer_streams(seed: int, K: int, T_fuel: float = 800.0, T_ox: float = 1500.0):
    """The two unmixed streams of cells_shear_layer (the same seeded draws): (T, Y [K]) of the
    fuel (Z = 1) and of the oxidiser (Z = 0), the ambient states far from the layer."""
    Y_fuel, Y_ox = _shear_streams(np.random.default_rng(seed), K)
    return (T_fuel, Y_fuel), (T_ox, Y_ox)


def cells_shear_layer(seed: int, K: int, nx: int = 256, ny: int = 256, delta: float = 8.0,
                      T_fuel: float = 800.0, T_ox: float = 1500.0):
    """2-D shear-layer field: Z = (1 + tanh(y/delta))/2 with a seeded sinusoidal displacement of
    5% of the height; T and Y mixed linearly in Z between two Dirichlet(1) streams (Z = 1 is fuel).
    Cells are ordered row-major (c = j*nx + i).  Returns T [n], Y [K, n], Z [n]."""
    rng = np.random.default_rng(seed)
    Y_fuel, Y_ox = _shear_streams(rng, K)
    m = int(rng.integers(1, 5))
    phi = rng.uniform(0.0, 2.0 * np.pi)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    y = (j - (ny - 1) / 2.0) + 0.05 * ny * np.sin(2.0 * np.pi * m * i / nx + phi)
    Z = (0.5 * (1.0 + np.tanh(y / delta))).ravel()
    T = Z * T_fuel + (1.0 - Z) * T_ox
    Y = Y_fuel[:, None] * Z[None, :] + Y_ox[:, None] * (1.0 - Z[None, :])
    return T, Y, Z


def workload_small():
    """10 species, 256 cells, T ~ U[1000, 1800] K, Dirichlet(1) Y, 1 atm, dt 1e-5 s."""
    mech = mechanism_small()
    T, Y = cells_uniform(101, mech.K, 256)
    return dict(name="mech10_256cells", mech=mech, p_Pa=1.0 * P_ATM_PA, T=T, Y=Y, dt=1e-5, rtol=1e-6, atol=1e-10)


def workload_shear_layer(n_side: int = 256):
    """53 species, 256x256 shear-layer field, 40 atm, dt 1e-5 s."""
    mech = mechanism_53()
    T, Y, _ = cells_shear_layer(102, mech.K, n_side, n_side)
    return dict(name=f"mech53_shear{n_side}x{n_side}", mech=mech, p_Pa=40.0 * P_ATM_PA, T=T, Y=Y, dt=1e-5,
                rtol=1e-6, atol=1e-10, streams=shear_layer_streams(102, mech.K))


def workload_0d(n: int = 608):
    """The 0D homogeneous-reactor stand-in of the paper's Fig. 2/3 ablation: the 53-species
    mechanism at 1200 K and 13.5 atm, one Dirichlet(1) mixture (seed 106) in n identical cells
    (repeated samples of one reactor), CFD step 1e-6 s."""
    mech = mechanism_53()
    rng = np.random.default_rng(106)
    Y1 = rng.dirichlet(np.ones(mech.K))
    T = np.full(n, 1200.0)
    Y = np.repeat(Y1[:, None], n, axis=1).copy()
    return dict(name=f"mech53_0d_reactor{n}", mech=mech, p_Pa=13.5 * P_ATM_PA, T=T, Y=Y, dt=1e-6, rtol=1e-6,
                atol=1e-10)


def workload_igniting(n: int = 16384):
    """53 species, igniting band T ~ U[1000, 1300] K, Dirichlet(1) Y, 20 atm, dt 1e-4 s."""
    mech = mechanism_53()
    T, Y = cells_uniform(105, mech.K, n, (1000.0, 1300.0))
    return dict(name=f"mech53_igniting{n}", mech=mech, p_Pa=20.0 * P_ATM_PA, T=T, Y=Y, dt=1e-4,
                rtol=1e-6, atol=1e-10)


def burnt_templates():
    """Equilibrium (T, Y) states of the 100-species mechanism at 60 atm, T in [2000, 2400] K
    (written by tests/golden/make_burnt_templates.py from the oracle's thermo)."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                        "burnt_templates_mech100.npz")
    d = np.load(path)
    return d["T"], d["Y"]


def cells_uneven(seed: int, K: int, n: int, order: str = "shuffled"):
    """Uneven-stiffness field: 10% igniting cells (T ~ U[900, 1200] K, two Dirichlet(1) streams
    mixed at Z ~ U[0.4, 0.6]), 60% cold cells (T ~ U[300, 700] K, Dirichlet(1) Y), 30% burnt
    cells (equilibrium templates).  order: "shuffled" or "blocked" (igniting, cold, burnt).
    Returns T [n], Y [K, n], class [n] (0 igniting, 1 cold, 2 burnt)."""
    rng = np.random.default_rng(seed)
    n_ign = n // 10
    n_burnt = (3 * n) // 10
    n_cold = n - n_ign - n_burnt
    Yf = rng.dirichlet(np.ones(K))
    Yo = rng.dirichlet(np.ones(K))
    Z = rng.uniform(0.4, 0.6, n_ign)
    T_ign = rng.uniform(900.0, 1200.0, n_ign)
    Y_ign = Yf[:, None] * Z[None, :] + Yo[:, None] * (1.0 - Z[None, :])
    T_cold = rng.uniform(300.0, 700.0, n_cold)
    Y_cold = rng.dirichlet(np.ones(K), size=n_cold).T
    Tt, Yt = burnt_templates()
    if Yt.shape[1] != K:
        raise ValueError("burnt templates are for the 100-species mechanism")
    pick = rng.integers(0, Tt.shape[0], n_burnt)
    T_b, Y_b = Tt[pick], Yt[pick].T
    T = np.concatenate([T_ign, T_cold, T_b])
    Y = np.concatenate([Y_ign, Y_cold, Y_b], axis=1)
    cls = np.concatenate([np.zeros(n_ign, np.int32), np.ones(n_cold, np.int32), np.full(n_burnt, 2, np.int32)])
    if order == "shuffled":
        perm = rng.permutation(n)
        T, Y, cls = T[perm], Y[:, perm], cls[perm]
    elif order != "blocked":
        raise ValueError("order must be 'shuffled' or 'blocked'")
    return T, np.ascontiguousarray(Y), cls


def workload_uneven(n: int = 262144, order: str = "shuffled"):
    """100 species / 700 reactions, uneven-stiffness field (igniting / cold / burnt), 60 atm,
    dt 5e-6 s."""
    mech = mechanism_100()
    T, Y, cls = cells_uneven(103, mech.K, n, order)
    return dict(name=f"mech100_uneven{n}_{order}", mech=mech, p_Pa=60.0 * P_ATM_PA, T=T, Y=Y, cls=cls, dt=5e-6,
                rtol=1e-6, atol=1e-10)
