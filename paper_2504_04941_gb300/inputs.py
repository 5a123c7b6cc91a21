"""Seeded synthetic inputs: reaction networks and initial cell states.

This module only *draws data*.  It holds none of the method's arithmetic: no rate
law, no Jacobian, no linear algebra and no time stepping.  Both the FP64 CPU oracle
and the CUDA path consume what it produces (a plain-text network file plus
structure-of-arrays cell arrays), and neither side imports the other.

Networks follow the ODE class of Sec. 2.2 (Eq. method-ode-thermochem): species
densities evolve by mass-action reactions with up to three reactants and three
products, each with a modified-Arrhenius coefficient

    k(T) = A * (T / T_ref)**b * exp(-theta / T)

(Sec. 2.2.1, item 1; the printed form repeats T_0, read here as a per-network
reference temperature T_ref and an activation temperature theta).  Reversible
reactions are written as two irreversible entries, as the paper's GRI-Mech
submechanism counts "116 elementary reactions (including inverse reactions)"
(Sec. 4.2).  When a network carries the temperature equation, each species has a
heat of formation h_s [J/mol] and a molar heat capacity cv_s [J/mol/K].

Workloads (seed = 250404941 + workload id):

1. ``robertson``   Robertson kinetics, 3 species, isothermal, 1024 cells.
2. ``combustion``  10 species / 2 elements / 30 reversible A+B<=>C+D reactions
                   with temperature, 65,536 cells.
3. ``ism``         32 species / 3 elements / 200 irreversible 1- and 2-body
                   reactions, isothermal, 1,048,576 cells.
4. ``robertson_mlp`` the Robertson network for the learned-guess study.
5. ``combined``    64 species / 4 elements / 500 reversible reactions with
                   temperature, 160^3 cells on Gaussian random fields.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 250404941
R_GAS = 8.314462618  # J / (mol K), CODATA 2018


# --------------------------------------------------------------------------- network


@dataclasses.dataclass
class Network:
    name: str
    species: List[str]
    elements: List[str]
    mass: np.ndarray          # [ns] g/mol
    h: np.ndarray             # [ns] J/mol heat of formation
    cv: np.ndarray            # [ns] J/(mol K)
    counts: np.ndarray        # [ns, ne] int, atoms of element e in species s
    energy: int               # 1: temperature equation, 0: isothermal
    t_ref: float
    t_min: float
    t_max: float
    reac_in: List[Tuple[int, ...]]
    reac_out: List[Tuple[int, ...]]
    A: np.ndarray             # [nr]
    b: np.ndarray             # [nr]
    theta: np.ndarray         # [nr] K
    pair: np.ndarray          # [nr] index of the reverse entry, -1 if none
    # temperature-dependent heat capacities (optional): cv_s(T) [J/(mol K)] =
    # sum_k cv_poly[s, 0, k] T^k below t_mid and sum_k cv_poly[s, 1, k] T^k from t_mid
    cv_poly: Optional[np.ndarray] = None     # [ns, 2, 5]
    t_mid: float = 1000.0
    # photo-reactions (Eq. photo-reaction-single): reaction -> cross-section sigma_r [cm^2]
    photo: Optional[Dict[int, float]] = None
    # tabulated rates (Sec. 2.2.1 item 3): grid (nT, T0, T1, nR, rho0, rho1), log-spaced,
    # and reaction -> ln k on it, shape [nR, nT]
    table_grid: Optional[Tuple[int, float, float, int, float, float]] = None
    tables: Optional[Dict[int, np.ndarray]] = None

    @property
    def ns(self) -> int:
        return len(self.species)

    @property
    def ne(self) -> int:
        return len(self.elements)

    @property
    def nr(self) -> int:
        return len(self.reac_in)

    @property
    def n(self) -> int:
        """Number of ODE unknowns (species, plus T when the energy equation is on)."""
        return self.ns + self.energy

    def to_text(self) -> str:
        out = ["kratos_network 1",
               f"name {self.name}",
               f"n_species {self.ns}",
               f"n_elements {self.ne}",
               f"n_reactions {self.nr}",
               f"energy {int(self.energy)}",
               f"t_ref {self.t_ref!r}",
               f"t_min {self.t_min!r}",
               f"t_max {self.t_max!r}",
               "elements " + " ".join(self.elements)]
        for s in range(self.ns):
            cnt = " ".join(str(int(c)) for c in self.counts[s])
            out.append(f"species {self.species[s]} {float(self.mass[s])!r} "
                       f"{float(self.h[s])!r} {float(self.cv[s])!r} {cnt}")
        for r in range(self.nr):
            ins = " ".join(str(i) for i in self.reac_in[r])
            outs = " ".join(str(i) for i in self.reac_out[r])
            out.append(f"reaction {len(self.reac_in[r])} {ins} {len(self.reac_out[r])} {outs} "
                       f"{float(self.A[r])!r} {float(self.b[r])!r} {float(self.theta[r])!r} "
                       f"{int(self.pair[r])}")
        if self.photo:
            out.append(f"photo {len(self.photo)}")
            for r, sg in sorted(self.photo.items()):
                out.append(f"ph {int(r)} {float(sg)!r}")
        if self.tables:
            nT, T0, T1, nR, R0, R1 = self.table_grid
            out.append(f"rate_table {int(nT)} {float(T0)!r} {float(T1)!r} {int(nR)} {float(R0)!r} "
                       f"{float(R1)!r} {len(self.tables)}")
            for r, tab in sorted(self.tables.items()):
                vals = " ".join(repr(float(v)) for v in np.asarray(tab, float).ravel())
                out.append(f"tab {int(r)} {vals}")
        if self.cv_poly is not None:
            out.append(f"cv_poly {float(self.t_mid)!r}")
            for sp in range(self.ns):
                co = " ".join(repr(float(c)) for c in np.asarray(self.cv_poly[sp]).ravel())
                out.append(f"cvp {sp} {co}")
        out.append("end")
        return "\n".join(out) + "\n"

    def write(self, path: str) -> str:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            f.write(self.to_text())
        return path


def _irreversible(name, species, elements, mass, h, cv, counts, energy, t_ref,
                  t_min, t_max, reactions) -> Network:
    """reactions: list of (ins, outs, A, b, theta, pair)."""
    return Network(
        name=name, species=list(species), elements=list(elements),
        mass=np.asarray(mass, float), h=np.asarray(h, float), cv=np.asarray(cv, float),
        counts=np.asarray(counts, np.int64).reshape(len(species), len(elements)),
        energy=int(energy), t_ref=float(t_ref), t_min=float(t_min), t_max=float(t_max),
        reac_in=[tuple(r[0]) for r in reactions], reac_out=[tuple(r[1]) for r in reactions],
        A=np.array([r[2] for r in reactions], float), b=np.array([r[3] for r in reactions], float),
        theta=np.array([r[4] for r in reactions], float),
        pair=np.array([r[5] for r in reactions], np.int64))


def with_nasa_heat_capacity(net: Network, seed: int = SEED_BASE + 6, t_mid: float = 1000.0) -> Network:
    """The network with temperature-dependent heat capacities in the two-range
    polynomial form of NASA-7 fits (Sec. 4.2: c_V rises above ~10^3 K as vibrational
    modes activate).  Synthetic coefficients: with u = (T - 300)/700,
        cv_s(T) = cv_s (1 + e_s (0.3 u^2 + 0.05 u^3 (1 - u)))   below t_mid = 1000 K,
        cv_s(T) = cv_s (1 + e_s (0.3 + 0.06 (T - 1000)/1000))   from t_mid,
    e_s ~ U(0.2, 1) (a 20-100 % rise by ~10^4 K; continuous at t_mid, positive for all
    T > 0), written out as monomial coefficients of T."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(0.2, 1.0, net.ns)
    P = np.polynomial.polynomial
    u = np.array([-300.0 / 700.0, 1.0 / 700.0])             # u(T) as a polynomial in T
    low_shape = P.polyadd(0.3 * P.polypow(u, 2), 0.05 * P.polymul(P.polypow(u, 3), P.polysub([1.0], u)))
    high_shape = np.array([0.3 - 0.06, 0.06 / 1000.0])      # 0.3 + 0.06 (T - 1000)/1000
    poly = np.zeros((net.ns, 2, 5))
    for sp in range(net.ns):
        lo = P.polyadd([1.0], e[sp] * low_shape) * net.cv[sp]
        hi = P.polyadd([1.0], e[sp] * high_shape) * net.cv[sp]
        poly[sp, 0, :len(lo)] = lo
        poly[sp, 1, :len(hi)] = hi
    return dataclasses.replace(net, name=net.name + "_nasa", cv_poly=poly, t_mid=float(t_mid))


def with_tabulated_rates(net: Network, frac: float, seed: int, nT: int = 33, nR: int = 9,
                         T_range=(5.0, 2.0e5), rho_range=(1e-5, 1e9)) -> Network:
    """A fraction of the two-body reactions switched to tabulated rates: ln k on a
    log-spaced (T, rho) grid, sampled from the reaction's own modified-Arrhenius law
    times a density factor rho^c_r, c_r ~ U(-0.3, 0.3) (a stand-in for the
    density-dependent rates the paper tabulates, e.g. falloff or escape probabilities;
    Sec. 2.2.1 item 3).  The Arrhenius parameters stay in the file but are not used."""
    rng = np.random.default_rng(seed)
    two = [r for r in range(net.nr) if len(net.reac_in[r]) == 2 and (not net.photo or r not in net.photo)]
    pick = sorted(rng.choice(two, max(1, int(round(frac * len(two)))), replace=False).tolist())
    Tn = np.geomspace(T_range[0], T_range[1], nT)
    Rn = np.geomspace(rho_range[0], rho_range[1], nR)
    tables = {}
    for r in pick:
        c = rng.uniform(-0.3, 0.3)
        lnk = (math.log(net.A[r]) + net.b[r] * np.log(Tn / net.t_ref) - net.theta[r] / Tn)
        tables[int(r)] = lnk[None, :] + c * np.log(Rn)[:, None]
    return dataclasses.replace(net, name=net.name + "_tab", tables=tables,
                               table_grid=(nT, T_range[0], T_range[1], nR, rho_range[0], rho_range[1]))


def with_photo_reactions(net: Network, seed: int) -> Network:
    """Every one-body reaction becomes a photo-reaction with cross-section
    sigma_r ~ log-uniform(1e-19, 1e-17) cm^2; its rate is F sigma_r (1 - e^-tau)/tau
    with the cell's flux factor F and optical depth tau (Eq. photo-reaction-single)."""
    rng = np.random.default_rng(seed)
    one = [r for r in range(net.nr) if len(net.reac_in[r]) == 1]
    photo = {int(r): float(10.0 ** rng.uniform(-19.0, -17.0)) for r in one}
    return dataclasses.replace(net, name=net.name + "_rad", photo=photo)


def radiation_fields(ncells: int, seed: int, flux_range=(1e6, 1e10), path_range=(1e13, 1e17)):
    """Per-cell photo flux factor F [cm^-2 s^-1] and path length dl [cm], log-uniform."""
    rng = np.random.default_rng(seed)
    F = np.exp(rng.uniform(math.log(flux_range[0]), math.log(flux_range[1]), ncells))
    dl = np.exp(rng.uniform(math.log(path_range[0]), math.log(path_range[1]), ncells))
    return F, dl


def robertson_network() -> Network:
    """Robertson's three-species stiff kinetics (k1=0.04, k2=3e7, k3=1e4), isothermal.

    y1 -> y2 (k1);  y2 + y2 -> y2 + y3 (k2);  y2 + y3 -> y1 + y3 (k3).
    One pseudo-element counted once in every species, so y1+y2+y3 is conserved.
    """
    rx = [((0,), (1,), 0.04, 0.0, 0.0, -1),
          ((1, 1), (1, 2), 3.0e7, 0.0, 0.0, -1),
          ((1, 2), (0, 2), 1.0e4, 0.0, 0.0, -1)]
    return _irreversible("robertson", ["Y1", "Y2", "Y3"], ["X"], [1.0, 1.0, 1.0],
                         [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [[1], [1], [1]], 0,
                         1.0, 1.0, 1.0e5, rx)


def decay_chain_network(k1: float, k2: float) -> Network:
    """Linear chain A -> B -> C (first-order, Sec. 2.2 B^i_j terms only)."""
    rx = [((0,), (1,), k1, 0.0, 0.0, -1), ((1,), (2,), k2, 0.0, 0.0, -1)]
    return _irreversible("decay_chain", ["A", "B", "C"], ["X"], [1.0, 1.0, 1.0],
                         [0.0] * 3, [0.0] * 3, [[1], [1], [1]], 0, 1.0, 1.0, 1.0e5, rx)


K_B_EV = 8.617333262e-5  # eV / K
I_H_EV = 13.6            # eV, ionisation energy of hydrogen (Sec. 4.3)


def stromgren_network(photo_rate: float) -> Network:
    """H / H+ / e- network of the Stromgren test (Sec. 4.3, Eqs. strom-chem, thermo-strom).

    photoionisation  H -> H+ + e-            rate photo_rate = F*sigma  [1/s]
    collisional ion. H + e- -> H+ + 2e-      k_ci = 1.05e-9 (T/300)^0.5 exp(-I_H/k_B T) cm^3/s
    recombination    H+ + e- -> H            alpha = 3.5e-12 (T/300)^-0.75 cm^3/s
    Elements: hydrogen nuclei and charge (e- carries -1, H+ carries +1).
    Isothermal (the equilibrium pin fixes T).
    """
    theta_ci = I_H_EV / K_B_EV
    rx = [((0,), (1, 2), float(photo_rate), 0.0, 0.0, -1),
          ((0, 2), (1, 2, 2), 1.05e-9, 0.5, theta_ci, -1),
          ((1, 2), (0,), 3.5e-12, -0.75, 0.0, -1)]
    return _irreversible("stromgren", ["H", "Hp", "e"], ["H", "Q"], [1.00794, 1.00739, 0.00055],
                         [0.0] * 3, [0.0] * 3, [[1, 0], [1, 1], [0, -1]], 0,
                         300.0, 1.0, 1.0e9, rx)


def _connected(ns: int, reactions: Sequence[Tuple[Tuple[int, ...], Tuple[int, ...]]]) -> bool:
    parent = list(range(ns))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ins, outs in reactions:
        sp = list(ins) + list(outs)
        for s in sp[1:]:
            parent[find(s)] = find(sp[0])
    roots = {find(s) for s in range(ns)}
    return len(roots) == 1


def _reversible_pairs_to_entries(pairs, A, b, theta, h):
    """Expand reversible reactions into forward/reverse irreversible entries.

    Both directions share A and b.  The endothermic direction carries the extra
    activation temperature |dH|/R, so k_f / k_r = exp(-dH_r / (R T)) (zero entropy
    change, equal mole numbers): detailed balance holds exactly at equilibrium.
    """
    rx = []
    for q, (ins, outs) in enumerate(pairs):
        dH = float(sum(h[o] for o in outs) - sum(h[i] for i in ins))
        th_f = float(theta[q]) + max(0.0, dH) / R_GAS
        th_r = float(theta[q]) + max(0.0, -dH) / R_GAS
        f_idx = len(rx)
        rx.append((tuple(ins), tuple(outs), float(A[q]), float(b[q]), th_f, f_idx + 1))
        rx.append((tuple(outs), tuple(ins), float(A[q]), float(b[q]), th_r, f_idx))
    return rx


def _bimolecular_pairs(comp: np.ndarray, n_pairs: int, rng: np.random.Generator,
                       max_tries: int = 200):
    """Draw n_pairs distinct element-conserving A+B <=> C+D reactions connecting all species."""
    ns = comp.shape[0]
    groups: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
    for i in range(ns):
        for j in range(i, ns):
            key = tuple((comp[i] + comp[j]).tolist())
            groups.setdefault(key, []).append((i, j))
    cands = []
    for key, plist in groups.items():
        for p, q in itertools.combinations(plist, 2):
            if set(p) & set(q):
                continue
            cands.append((p, q))
    if len(cands) < n_pairs:
        raise ValueError(f"only {len(cands)} candidate reactions for {n_pairs} requested")
    for _ in range(max_tries):
        pick = rng.choice(len(cands), size=n_pairs, replace=False)
        chosen = [cands[k] for k in sorted(pick)]
        chosen = [(p, q) if rng.random() < 0.5 else (q, p) for p, q in chosen]
        if _connected(ns, chosen):
            return chosen
    raise RuntimeError("could not draw a connected reaction set")


def combustion_network(seed: int = SEED_BASE + 2, n_species: int = 10, n_elements: int = 2,
                       n_reversible: int = 30, name: str = "combustion10") -> Network:
    """Synthetic combustion-like network with temperature equation.

    Species: the n_elements atoms plus compositions drawn (without replacement) from
    element-count vectors with each count <= 3 and 2..4 atoms in total.  Element
    masses 1, 16, 12, 14 g/mol.  Reactions: distinct element-conserving
    A+B <=> C+D, log10 A ~ U(8,14) [cm^3 mol^-1 s^-1], b ~ U(-1,1), theta ~ U(0,3e4) K,
    heats of formation ~ U(-3e5, 3e5) J/mol, T_ref = 1 K.  cv_s = 1.5 R for atoms,
    2.5 R for diatomics and 3 R otherwise.
    """
    rng = np.random.default_rng(seed)
    elem_names = ["H", "O", "C", "N"][:n_elements]
    elem_mass = np.array([1.0, 16.0, 12.0, 14.0][:n_elements])
    atoms = [tuple(int(i == e) for i in range(n_elements)) for e in range(n_elements)]
    pool = [c for c in itertools.product(range(4), repeat=n_elements)
            if 2 <= sum(c) <= 4]
    pool.sort()
    need = n_species - n_elements
    if need > len(pool):
        raise ValueError("not enough compositions")
    for _ in range(200):
        pick = rng.choice(len(pool), size=need, replace=False)
        comps = atoms + [pool[k] for k in sorted(pick)]
        comp = np.array(comps, np.int64)
        try:
            pairs = _bimolecular_pairs(comp, n_reversible, rng)
            break
        except (ValueError, RuntimeError):
            continue
    else:
        raise RuntimeError("could not build combustion network")
    logA = rng.uniform(8.0, 14.0, n_reversible)
    b = rng.uniform(-1.0, 1.0, n_reversible)
    theta = rng.uniform(0.0, 3.0e4, n_reversible)
    h = rng.uniform(-3.0e5, 3.0e5, n_species)
    natoms = comp.sum(axis=1)
    cv = np.where(natoms == 1, 1.5, np.where(natoms == 2, 2.5, 3.0)) * R_GAS
    mass = comp @ elem_mass
    names = ["".join(f"{elem_names[e]}{c if c > 1 else ''}" for e, c in enumerate(row) if c)
             for row in comps]
    names = [f"{nm}_{s}" for s, nm in enumerate(names)]
    rx = _reversible_pairs_to_entries(pairs, 10.0 ** logA, b, theta, h)
    return _irreversible(name, names, elem_names, mass, h, cv, comp, 1, 1.0, 10.0, 1.0e5, rx)


def ism_network(seed: int = SEED_BASE + 3, n_species: int = 32, n_reactions: int = 200,
                frac_activated: float = 0.5, frac_one_body: float = 0.3) -> Network:
    """Synthetic ISM-like network, isothermal, irreversible reactions (UMIST-like form).

    32 species over H, C, O (each count <= 3, 1..5 atoms), 200 reactions:
    a fraction ``frac_one_body`` are 1-body A -> B + C (photo / cosmic-ray, constant
    rate), the rest 2-body A + B -> C (+ D).  All rates log10 k(300 K) ~ U(-18,-9)
    (s^-1 or cm^3 s^-1).  2-body: b ~ U(-1,1); a fraction ``frac_activated`` has
    theta ~ U(0, 3e4) K, the rest theta = 0.  T_ref = 300 K.
    """
    rng = np.random.default_rng(seed)
    ne = 3
    elem_names = ["H", "C", "O"]
    elem_mass = np.array([1.0, 12.0, 16.0])
    atoms = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    pool = sorted(c for c in itertools.product(range(4), repeat=ne) if 2 <= sum(c) <= 5)
    pick = rng.choice(len(pool), size=n_species - ne, replace=False)
    comps = atoms + [pool[k] for k in sorted(pick)]
    comp = np.array(comps, np.int64)
    ns = n_species
    # candidate 2-body A+B -> C (+D) and 1-body A -> B + C
    by_comp: Dict[Tuple[int, ...], List[int]] = {}
    for s in range(ns):
        by_comp.setdefault(tuple(comp[s].tolist()), []).append(s)
    pairs_by_sum: Dict[Tuple[int, ...], List[Tuple[int, int]]] = {}
    for i in range(ns):
        for j in range(i, ns):
            pairs_by_sum.setdefault(tuple((comp[i] + comp[j]).tolist()), []).append((i, j))
    two_body, one_body = [], []
    for i in range(ns):
        for j in range(i, ns):
            key = tuple((comp[i] + comp[j]).tolist())
            for c in by_comp.get(key, []):
                two_body.append(((i, j), (c,)))
            for (c, d) in pairs_by_sum.get(key, []):
                if {c, d} != {i, j} and not ({c, d} & {i, j}):
                    two_body.append(((i, j), (c, d)))
    for a in range(ns):
        for (c, d) in pairs_by_sum.get(tuple(comp[a].tolist()), []):
            if a not in (c, d):
                one_body.append(((a,), (c, d)))
    n1 = int(round(frac_one_body * n_reactions))
    n2 = n_reactions - n1
    for _ in range(500):
        p1 = rng.choice(len(one_body), size=min(n1, len(one_body)), replace=False)
        p2 = rng.choice(len(two_body), size=n2 + (n1 - len(p1)), replace=False)
        chosen = [one_body[k] for k in sorted(p1)] + [two_body[k] for k in sorted(p2)]
        if _connected(ns, chosen):
            break
    else:
        raise RuntimeError("could not build ism network")
    rx = []
    for ins, outs in chosen:
        logk = rng.uniform(-18.0, -9.0)
        if len(ins) == 1:
            rx.append((ins, outs, 10.0 ** logk, 0.0, 0.0, -1))
        else:
            b = rng.uniform(-1.0, 1.0)
            th = rng.uniform(0.0, 3.0e4) if rng.random() < frac_activated else 0.0
            # UMIST convention: the prefactor alpha = A is drawn, k(300 K) = A exp(-theta/300)
            rx.append((ins, outs, 10.0 ** logk, b, th, -1))
    names = ["".join(f"{elem_names[e]}{c if c > 1 else ''}" for e, c in enumerate(row) if c)
             for row in comps]
    names = [f"{nm}_{s}" for s, nm in enumerate(names)]
    mass = comp @ elem_mass
    return _irreversible("ism32", names, elem_names, mass, np.zeros(ns), np.zeros(ns), comp, 0,
                         300.0, 10.0, 1.0e5, rx)


# --------------------------------------------------------------------------- cells


@dataclasses.dataclass
class Cells:
    y: np.ndarray    # [ns, ncells] SoA, float64
    T: np.ndarray    # [ncells]
    rho: np.ndarray  # [ncells]
    # photo-reactions (Eq. photo-reaction-single): flux factor F = L dl / dV [cm^-2 s^-1]
    # and path length dl [cm] per cell; None: F = 1, dl = 0 (optically thin, k = sigma)
    flux: Optional[np.ndarray] = None
    path: Optional[np.ndarray] = None

    @property
    def ncells(self) -> int:
        return self.T.shape[0]

    def subset(self, idx) -> "Cells":
        idx = np.asarray(idx)
        pick = lambda a: None if a is None else a[idx].copy()
        return Cells(np.ascontiguousarray(self.y[:, idx]), self.T[idx].copy(), self.rho[idx].copy(),
                     pick(self.flux), pick(self.path))


def robertson_cells(ncells: int, seed: int = SEED_BASE + 1) -> Cells:
    """y1 ~ U(0.9, 1), y2 = 0, y3 = 1 - y1; T = 300 K and rho = 1 (unused, isothermal)."""
    rng = np.random.default_rng(seed)
    y1 = rng.uniform(0.9, 1.0, ncells)
    y = np.stack([y1, np.zeros(ncells), 1.0 - y1])
    return Cells(np.ascontiguousarray(y), np.full(ncells, 300.0), np.ones(ncells))


def combustion_cells(net: Network, ncells: int, seed: int = SEED_BASE + 2,
                     t_range=(900.0, 2500.0), log_rho_range=(-4.0, -1.0),
                     T: Optional[np.ndarray] = None, log_rho: Optional[np.ndarray] = None) -> Cells:
    """T ~ U(900,2500) K, log10 rho ~ U(-4,-1) g/cm^3, mass fractions ~ Dirichlet(1);
    n_s = rho * Y_s / W_s [mol/cm^3].  T and log10 rho may be supplied (random fields)."""
    rng = np.random.default_rng(seed)
    if T is None:
        T = rng.uniform(*t_range, ncells)
    if log_rho is None:
        log_rho = rng.uniform(*log_rho_range, ncells)
    rho = 10.0 ** np.asarray(log_rho, float)
    Y = rng.dirichlet(np.ones(net.ns), size=ncells).T            # [ns, ncells]
    y = rho[None, :] * Y / net.mass[:, None]
    return Cells(np.ascontiguousarray(y), np.asarray(T, float).copy(), rho)


def ism_cells(net: Network, ncells: int, seed: int = SEED_BASE + 3,
              t_range=(10.0, 1.0e4), nh_range=(1.0, 1.0e8)) -> Cells:
    """T log-uniform 10 K..1e4 K, n_H log-uniform 1..1e8 cm^-3; abundances
    n_s = n_H * f_s with f ~ Dirichlet(1) (number densities, cm^-3); rho = n_H."""
    rng = np.random.default_rng(seed)
    T = np.exp(rng.uniform(math.log(t_range[0]), math.log(t_range[1]), ncells))
    nH = np.exp(rng.uniform(math.log(nh_range[0]), math.log(nh_range[1]), ncells))
    f = rng.dirichlet(np.ones(net.ns), size=ncells).T
    y = nH[None, :] * f
    return Cells(np.ascontiguousarray(y), T, nH)


def gaussian_random_field(n: int, slope: float, seed: int) -> np.ndarray:
    """Seeded periodic Gaussian random field on n^3, power spectrum ~ k^slope, standardised."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    fk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n)[:, None, None]
    ky = np.fft.fftfreq(n)[None, :, None]
    kz = np.fft.rfftfreq(n)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    nz = kk > 0
    amp[nz] = kk[nz] ** (slope / 2.0)
    g = np.fft.irfftn(fk * amp, s=(n, n, n), axes=(0, 1, 2))
    g = (g - g.mean()) / g.std()
    return g.reshape(-1)


def _normal_cdf(x: np.ndarray) -> np.ndarray:
    from scipy.special import ndtr
    return ndtr(x)


def combined_cells(net: Network, n_side: int = 160, seed: int = SEED_BASE + 5) -> Cells:
    """GRF T in 50..3000 K (log-uniform marginal) and log10 rho in -4..-1, slope -11/3."""
    T, log_rho = combined_fields(n_side, seed)
    return combustion_cells(net, n_side ** 3, seed=seed + 2000, T=T.ravel(), log_rho=log_rho.ravel())


def combined_fields(n_side: int = 160, seed: int = SEED_BASE + 5):
    """(T, log10 rho) of every cell of the n_side^3 Gaussian-random-field grid."""
    key = (n_side, seed)
    if key not in _FIELDS:
        g1 = gaussian_random_field(n_side, -11.0 / 3.0, seed)
        g2 = gaussian_random_field(n_side, -11.0 / 3.0, seed + 1000)
        _FIELDS.clear()
        _FIELDS[key] = (50.0 * 60.0 ** _normal_cdf(g1), -4.0 + 3.0 * _normal_cdf(g2))
    return _FIELDS[key]


_FIELDS: Dict[tuple, tuple] = {}


def combined_cells_sample(net: Network, n: int, seed: int = SEED_BASE + 5, n_side: int = 160) -> Cells:
    """n cells drawn without replacement (seeded) from the n_side^3 random-field grid of
    combined_cells: the same T and rho fields, compositions drawn as for the grid."""
    T, log_rho = combined_fields(n_side, seed)
    idx = np.sort(np.random.default_rng(seed + 3000).choice(n_side ** 3, n, replace=False))
    return combustion_cells(net, n, seed=seed + 2000, T=T.ravel()[idx], log_rho=log_rho.ravel()[idx])


# --------------------------------------------------------------------------- workloads


@dataclasses.dataclass
class Tolerances:
    dt: float
    rtol: float
    atol: float
    h_init: float
    h_min: float
    atol_mode: int = 0        # 0 absolute; 1 scaled by the cell's initial total of element 0
    max_substeps: int = 100000
    max_newton: int = 8


@dataclasses.dataclass
class Workload:
    wid: int
    name: str
    network: Network
    cells: Cells
    tol: Tolerances


FULL_CELLS = {1: 1024, 2: 65536, 3: 1048576, 4: 262144, 5: 160 ** 3, 6: 65536, 7: 65536, 8: 65536}


def tolerances(wid: int) -> Tolerances:
    if wid in (1, 4):
        return Tolerances(dt=1.0e4, rtol=1e-6, atol=1e-10, h_init=1e-6, h_min=1e-24)
    if wid in (2, 6, 8):
        return Tolerances(dt=1.0e-6, rtol=1e-6, atol=1e-20, h_init=1e-12, h_min=1e-30)
    if wid == 7:
        return Tolerances(dt=1.0e10, rtol=1e-6, atol=1e-10, h_init=1e-2, h_min=1e-20,
                          atol_mode=1)
    if wid == 5:
        # dt = 1e-6 s as for the 10-species network (the workload gives none)
        return Tolerances(dt=1.0e-6, rtol=1e-6, atol=1e-20, h_init=1e-13, h_min=1e-30)
    if wid == 3:
        return Tolerances(dt=1.0e10, rtol=1e-6, atol=1e-10, h_init=1e-2, h_min=1e-20,
                          atol_mode=1)
    raise ValueError(wid)


def network(wid: int) -> Network:
    if wid in (1, 4):
        return robertson_network()
    if wid == 2:
        return combustion_network()
    if wid == 3:
        return ism_network()
    if wid == 5:
        return combustion_network(seed=SEED_BASE + 5, n_species=64, n_elements=4,
                                  n_reversible=500, name="combined64")
    if wid == 6:
        return with_nasa_heat_capacity(combustion_network())
    if wid == 7:
        return with_tabulated_rates(with_photo_reactions(ism_network(), SEED_BASE + 70), 0.3, SEED_BASE + 71)
    if wid == 8:
        return with_tabulated_rates(combustion_network(), 0.2, SEED_BASE + 80)
    raise ValueError(wid)


def workload(wid: int, ncells: Optional[int] = None, seed: Optional[int] = None) -> Workload:
    """Network, seeded cells and tolerances of workload ``wid`` (1..5).

    ``ncells`` < full size draws the first cells of the same seeded stream shape
    (a smaller, independent draw with the same distributions)."""
    net = network(wid)
    s = SEED_BASE + wid if seed is None else seed
    n = FULL_CELLS[wid] if ncells is None else int(ncells)
    if wid in (1, 4):
        cells = robertson_cells(n, s)
    elif wid in (2, 6, 8):
        cells = combustion_cells(net, n, SEED_BASE + 2 if seed is None else seed)
    elif wid == 7:
        cells = ism_cells(net, n, SEED_BASE + 3 if seed is None else seed)
        cells.flux, cells.path = radiation_fields(n, s + 1)
    elif wid == 3:
        cells = ism_cells(net, n, s)
    elif wid == 5:
        if n >= 160 ** 3:
            cells = combined_cells(net, 160, s)
        else:
            cells = combined_cells_sample(net, n, s)
    names = {1: "robertson", 2: "combustion10", 3: "ism32", 4: "robertson_mlp", 5: "combined64",
             6: "combustion10_nasa", 7: "ism32_rad", 8: "combustion10_tab"}
    return Workload(wid, names[wid], net, cells, tolerances(wid))
