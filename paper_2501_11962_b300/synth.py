"""Seeded synthetic molecular systems and discretised paths.

This module builds inputs only: topology, force-field parameters, box and bead
coordinates.  It evaluates no potential, force, Hessian or effective potential;
the CUDA path and the FP64 checker both consume what it returns.

The five workloads stand in for the 151,850-atom membrane-protein system of the
paper's benchmarks (Appendix A.1), which is not available.  They are:

  1. 256 Lennard-Jones argon atoms on an fcc lattice, reduced density 0.8,
     rc = 1.0 nm, N = 16 beads, FP64 arithmetic.
  2. 1,000 flexible three-site waters at 1 g/cm^3, rc = 0.9 nm, N = 64.
  3. 8,000 waters at 1 g/cm^3, rc = 1.0 nm, N = 128.
  4. 3,333 waters plus one neutral ion, rc = 1.0 nm, eight paths of
     N = 24 ... 256 beads, with a two-group centroid-distance CV for the bias.
  5. 600 bonded 50-atom chains plus 40,000 waters in an 11.5 nm box
     (Q = 150,000), rc = 1.0 nm, N = 64.

Every bead is the base structure plus independent N(0, 0.01 nm) displacements,
rounded to float32 once; both sides read the same float32 values.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# u per nm^3 in one g/cm^3 (Avogadro's number times 1e-21 cm^3 per nm^3)
_U_PER_NM3_PER_G_CM3 = 602.214076

CUTOFF_SHIFTED_FORCE = 0
CUTOFF_POT_SHIFT = 1


@dataclass
class System:
    """Topology and parameters of one periodic system (units: nm, ps, u, e, kJ/mol)."""

    box: np.ndarray                      # (3,) float64, rectangular box edges
    type: np.ndarray                     # (Q,) int32 atom type
    lj_sigma: np.ndarray                 # (n_types,) float64
    lj_eps: np.ndarray                   # (n_types,) float64
    charge: np.ndarray                   # (Q,) float64, e
    mass: np.ndarray                     # (Q,) float64, u
    mol_id: np.ndarray                   # (Q,) int32
    mol_local: np.ndarray                # (Q,) int32 position inside its molecule
    bond_ij: np.ndarray                  # (n_bonds, 2) int32
    bond_r0: np.ndarray                  # (n_bonds,) float64
    bond_k: np.ndarray                   # (n_bonds,) float64
    angle_ijk: np.ndarray                # (n_angles, 3) int32, j is the vertex
    angle_th0: np.ndarray                # (n_angles,) float64, rad
    angle_k: np.ndarray                  # (n_angles,) float64
    rc: float = 1.0
    eps_rf: float = 78.0
    cutoff_mode: int = CUTOFF_SHIFTED_FORCE
    dt_path: float = 0.002               # ps, time step of the discretised path
    nu_path: float = 5.0                 # 1/ps, friction of the path action
    temperature: float = 300.0           # K
    elec: int = 0                        # ELEC_RF, or ELEC_PME (Ewald: real space + SPME)
    ew_beta: float = 0.0                 # 1/nm, Ewald splitting parameter (ELEC_PME)
    pme_grid: tuple = (0, 0, 0)          # SPME grid points per box edge (ELEC_PME)
    pme_order: int = 4                   # B-spline order of the SPME (ELEC_PME)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.type.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.lj_sigma.shape[0])


ELEC_RF, ELEC_PME = 0, 1


def _nice_fft_size(n: int) -> int:
    """Smallest m >= n whose prime factors are 2, 3 and 5."""
    m = max(int(n), 1)
    while True:
        k = m
        for f in (2, 3, 5):
            while k % f == 0:
                k //= f
        if k == 1:
            return m
        m += 1


def with_pme(system: System, spacing: float = 0.12, rtol: float = 1e-5, order: int = 4) -> System:
    """A copy of `system` with Ewald electrostatics: beta from erfc(beta rc) = rtol (bisection)
    and an SPME grid of at most `spacing` nm (FFT-friendly sizes), B-splines of `order`."""
    from math import erfc
    lo, hi = 0.0, 100.0 / system.rc
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if erfc(mid * system.rc) > rtol:
            lo = mid
        else:
            hi = mid
    grid = tuple(_nice_fft_size(int(np.ceil(system.box[d] / spacing))) for d in range(3))
    import dataclasses
    return dataclasses.replace(system, elec=ELEC_PME, ew_beta=hi, pme_grid=grid, pme_order=order)


@dataclass
class Workload:
    system: System
    paths: list                  # list of float32 arrays, each (N_p, Q, 3)
    precision: str = "mixed"     # "mixed" (FP32 pair math) or "fp64"
    fd_h: float = 1e-5
    cv_groups: tuple | None = None   # (group A indices, group B indices) for the bias
    bias: dict | None = None
    label: str = ""


# ----------------------------------------------------------------------------------------
# small geometry helpers (no physics)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from random unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random((3, n))
    q = np.stack([
        np.sqrt(1 - u1) * np.sin(2 * np.pi * u2),
        np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
        np.sqrt(u1) * np.sin(2 * np.pi * u3),
        np.sqrt(u1) * np.cos(2 * np.pi * u3),
    ], axis=1)
    x, y, z, w = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _water_template(r0: float = 0.1, theta_deg: float = 109.47) -> np.ndarray:
    """O, H1, H2 coordinates of a water at its ideal geometry, O at the origin."""
    half = np.deg2rad(theta_deg) / 2
    return np.array([
        [0.0, 0.0, 0.0],
        [r0 * np.sin(half), 0.0, r0 * np.cos(half)],
        [-r0 * np.sin(half), 0.0, r0 * np.cos(half)],
    ])


def _lattice_sites(n_side: tuple, box: np.ndarray) -> np.ndarray:
    g = [np.arange(n) * (box[d] / n) + 0.5 * box[d] / n for d, n in enumerate(n_side)]
    return np.stack(np.meshgrid(*g, indexing="ij"), axis=-1).reshape(-1, 3)


# ----------------------------------------------------------------------------------------
# parameter blocks

WATER_O = dict(sigma=0.3166, eps=0.65, q=-0.8476, m=15.999)
WATER_H = dict(sigma=0.0, eps=0.0, q=0.4238, m=1.008)
WATER_BOND = dict(r0=0.1, k=345000.0)
WATER_ANGLE = dict(th0_deg=109.47, k=383.0)
ION = dict(sigma=0.3166, eps=0.65, q=0.0, m=22.99)
CHAIN = dict(sigma=0.35, eps=0.3, m=12.011, q_std=0.3, bond_r0=0.15, bond_k=345000.0,
             angle_deg=111.0, angle_k=383.0)


class _Builder:
    """Accumulates atoms, molecules, bonds and angles."""

    def __init__(self):
        self.pos, self.type, self.q, self.m, self.mol, self.loc = [], [], [], [], [], []
        self.bonds, self.b_r0, self.b_k = [], [], []
        self.angles, self.a_th0, self.a_k = [], [], []
        self.n_mol = 0
        self.n = 0

    def add_molecule(self, pos, types, q, m, bonds=(), angles=()):
        base = self.n
        k = len(pos)
        self.pos.append(np.asarray(pos, dtype=np.float64))
        self.type.append(np.asarray(types, dtype=np.int32))
        self.q.append(np.asarray(q, dtype=np.float64))
        self.m.append(np.asarray(m, dtype=np.float64))
        self.mol.append(np.full(k, self.n_mol, dtype=np.int32))
        self.loc.append(np.arange(k, dtype=np.int32))
        self.n += k
        for (i, j, r0, kk) in bonds:
            self.bonds.append((base + i, base + j))
            self.b_r0.append(r0)
            self.b_k.append(kk)
        for (i, j, l, th0, kk) in angles:
            self.angles.append((base + i, base + j, base + l))
            self.a_th0.append(th0)
            self.a_k.append(kk)
        self.n_mol += 1

    def add_waters(self, o_pos: np.ndarray, rng: np.random.Generator, t_o: int, t_h: int):
        tmpl = _water_template(WATER_BOND["r0"], WATER_ANGLE["th0_deg"])
        rots = _random_rotations(rng, len(o_pos))
        th0 = np.deg2rad(WATER_ANGLE["th0_deg"])
        for c, R in zip(o_pos, rots):
            xyz = c + tmpl @ R.T
            self.add_molecule(
                xyz, [t_o, t_h, t_h],
                [WATER_O["q"], WATER_H["q"], WATER_H["q"]],
                [WATER_O["m"], WATER_H["m"], WATER_H["m"]],
                bonds=[(0, 1, WATER_BOND["r0"], WATER_BOND["k"]), (0, 2, WATER_BOND["r0"], WATER_BOND["k"])],
                angles=[(1, 0, 2, th0, WATER_ANGLE["k"])])

    def finish(self, box, sigma, eps, **kw):
        def cat(xs, dt):
            return np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
        sys = System(
            box=np.asarray(box, dtype=np.float64),
            type=cat(self.type, np.int32),
            lj_sigma=np.asarray(sigma, dtype=np.float64),
            lj_eps=np.asarray(eps, dtype=np.float64),
            charge=cat(self.q, np.float64),
            mass=cat(self.m, np.float64),
            mol_id=cat(self.mol, np.int32),
            mol_local=cat(self.loc, np.int32),
            bond_ij=np.asarray(self.bonds, dtype=np.int32).reshape(-1, 2),
            bond_r0=np.asarray(self.b_r0, dtype=np.float64),
            bond_k=np.asarray(self.b_k, dtype=np.float64),
            angle_ijk=np.asarray(self.angles, dtype=np.int32).reshape(-1, 3),
            angle_th0=np.asarray(self.a_th0, dtype=np.float64),
            angle_k=np.asarray(self.a_k, dtype=np.float64),
            **kw)
        return sys, np.concatenate(self.pos)


def water_box_edge(n_waters: int, extra_mass: float = 0.0, density_g_cm3: float = 1.0) -> float:
    mass = n_waters * (WATER_O["m"] + 2 * WATER_H["m"]) + extra_mass
    return (mass / (density_g_cm3 * _U_PER_NM3_PER_G_CM3)) ** (1.0 / 3.0)


# ----------------------------------------------------------------------------------------
# systems


def lj_fcc(n_cells: int = 4, sigma: float = 0.34, eps: float = 0.996, mass: float = 39.95,
           rho_reduced: float = 0.8, rc: float = 1.0):
    """Argon-like LJ atoms on an fcc lattice of n_cells^3 unit cells (4 atoms each)."""
    q_atoms = 4 * n_cells ** 3
    vol = q_atoms * sigma ** 3 / rho_reduced
    L = vol ** (1.0 / 3.0)
    a = L / n_cells
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(*[np.arange(n_cells)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) + 0.25) * a
    sys = System(
        box=np.array([L, L, L]), type=np.zeros(q_atoms, np.int32),
        lj_sigma=np.array([sigma]), lj_eps=np.array([eps]),
        charge=np.zeros(q_atoms), mass=np.full(q_atoms, mass),
        mol_id=np.arange(q_atoms, dtype=np.int32), mol_local=np.zeros(q_atoms, np.int32),
        bond_ij=np.zeros((0, 2), np.int32), bond_r0=np.zeros(0), bond_k=np.zeros(0),
        angle_ijk=np.zeros((0, 3), np.int32), angle_th0=np.zeros(0), angle_k=np.zeros(0),
        rc=rc, eps_rf=1.0, name=f"lj_fcc_{q_atoms}")
    return sys, pos


def water_box(n_waters: int, rc: float, seed: int, n_ions: int = 0, eps_rf: float = 78.0,
              jitter: float = 0.02):
    """Flexible three-site waters (plus optional neutral ions) on a cubic lattice."""
    rng = np.random.default_rng(seed)
    L = water_box_edge(n_waters, extra_mass=n_ions * ION["m"])
    box = np.array([L, L, L])
    n_mol = n_waters + n_ions
    n_side = int(np.ceil(n_mol ** (1.0 / 3.0)))
    sites = _lattice_sites((n_side,) * 3, box)
    pick = rng.permutation(len(sites))[:n_mol]
    sites = sites[np.sort(pick)] + rng.normal(0.0, jitter, (n_mol, 3))
    ion_slots = set(rng.choice(n_mol, size=n_ions, replace=False).tolist()) if n_ions else set()
    b = _Builder()
    t_o, t_h, t_ion = 0, 1, 2
    water_sites = [s for k, s in enumerate(sites) if k not in ion_slots]
    b.add_waters(np.array(water_sites), rng, t_o, t_h)
    for k in sorted(ion_slots):
        b.add_molecule([sites[k]], [t_ion], [ION["q"]], [ION["m"]])
    sigma = [WATER_O["sigma"], WATER_H["sigma"]] + ([ION["sigma"]] if n_ions else [])
    eps = [WATER_O["eps"], WATER_H["eps"]] + ([ION["eps"]] if n_ions else [])
    sys, pos = b.finish(box, sigma, eps, rc=rc, eps_rf=eps_rf,
                        name=f"water_{n_waters}" + (f"_ion{n_ions}" if n_ions else ""))
    return sys, pos


def _grid_neighbors(grid, counts, cell, ncell):
    """Atom ids stored in the 27 cells around `cell` (periodic)."""
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                c = ((cell[0] + dx) % ncell[0], (cell[1] + dy) % ncell[1], (cell[2] + dz) % ncell[2])
                k = counts[c]
                if k:
                    out.append(grid[c][:k])
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def chains_and_water(n_chains: int = 600, chain_len: int = 50, n_waters: int = 40000,
                     box_edge: float = 11.5, rc: float = 1.0, seed: int = 1005,
                     eps_rf: float = 78.0, min_sep: float = 0.2, water_clear: float = 0.22):
    """Bonded chains (self-avoiding walks with fixed bond and angle) in a water bath.

    The chains are grown first: bond length 0.15 nm, bond angle 111 deg, uniform
    random dihedral, and every new atom kept at least `min_sep` from all earlier
    chain atoms except its two predecessors.  Waters then occupy lattice sites
    whose oxygen is at least `water_clear` from every chain atom.
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    L = float(box_edge)
    box = np.array([L, L, L])
    ncell = tuple(int(L // min_sep) for _ in range(3))
    kmax = 16
    grid = np.zeros(ncell + (kmax,), dtype=np.int64)
    counts = np.zeros(ncell, dtype=np.int64)
    placed = []
    edge = L / np.array(ncell)

    def cell_of(p):
        w = np.mod(p, L)
        return tuple(np.minimum((w / edge).astype(int), np.array(ncell) - 1))

    def ok(p, skip):
        ids = _grid_neighbors(grid, counts, cell_of(p), ncell)
        if len(ids):
            ids = ids[~np.isin(ids, skip)]
        if len(ids) == 0:
            return True
        d = np.asarray([placed[i] for i in ids]) - p
        d -= L * np.round(d / L)
        return bool(np.all(np.einsum("ij,ij->i", d, d) >= min_sep * min_sep))

    def insert(p):
        c = cell_of(p)
        if counts[c] >= kmax:
            return False
        grid[c][counts[c]] = len(placed)
        counts[c] += 1
        placed.append(p)
        return True

    def rollback(n_keep):
        while len(placed) > n_keep:
            pid = len(placed) - 1
            c = cell_of(placed[pid])
            row = grid[c][:counts[c]]
            keep = row[row != pid]
            counts[c] = len(keep)
            grid[c][:len(keep)] = keep
            placed.pop()

    b_len, theta = CHAIN["bond_r0"], np.deg2rad(CHAIN["angle_deg"])
    chains = []
    for _ in range(n_chains):
        for _attempt in range(200):
            start = len(placed)
            p0 = rng.random(3) * L
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            p1 = p0 + b_len * u
            if not (ok(p0, []) and insert(p0) and ok(p1, [start]) and insert(p1)):
                rollback(start)
                continue
            good = True
            for k in range(2, chain_len):
                a, bb = placed[start + k - 2], placed[start + k - 1]
                e = (bb - a) / np.linalg.norm(bb - a)
                t = rng.normal(size=3)
                t -= t.dot(e) * e
                t /= np.linalg.norm(t)
                for _t in range(60):
                    phi = rng.random() * 2 * np.pi
                    perp = np.cos(phi) * t + np.sin(phi) * np.cross(e, t)
                    d = np.cos(np.pi - theta) * e + np.sin(np.pi - theta) * perp
                    p = bb + b_len * d
                    if ok(p, [start + k - 1, start + k - 2]):
                        break
                else:
                    good = False
                    break
                if not insert(p):
                    good = False
                    break
            if good:
                chains.append([placed[start + k] for k in range(chain_len)])
                break
            rollback(start)
        else:
            raise RuntimeError("chain growth failed; lower the density")

    chain_xyz = [np.array(atoms) for atoms in chains]
    all_chain = np.concatenate(chain_xyz) if chain_xyz else np.zeros((0, 3))

    # water sites on the coarsest lattice that leaves enough free sites
    tree = cKDTree(np.mod(all_chain, L), boxsize=L) if len(all_chain) else None
    n_side = int(np.ceil(n_waters ** (1.0 / 3.0)))
    while True:
        sites = _lattice_sites((n_side,) * 3, box)
        if tree is not None:
            dmin, _ = tree.query(np.mod(sites, L), k=1)
            free = sites[dmin >= water_clear]
        else:
            free = sites
        if len(free) >= n_waters:
            break
        n_side += 1
    pick = np.sort(rng.permutation(len(free))[:n_waters])
    o_pos = free[pick]

    bld = _Builder()
    t_c, t_o, t_h = 0, 1, 2
    th_c = np.deg2rad(CHAIN["angle_deg"])
    for xyz in chain_xyz:
        # keep the chain whole; put its first atom inside the box
        xyz = xyz - L * np.floor(xyz[0] / L)
        q = rng.normal(0.0, CHAIN["q_std"], chain_len)
        q -= q.mean()
        bonds = [(k, k + 1, CHAIN["bond_r0"], CHAIN["bond_k"]) for k in range(chain_len - 1)]
        angles = [(k, k + 1, k + 2, th_c, CHAIN["angle_k"]) for k in range(chain_len - 2)]
        bld.add_molecule(xyz, [t_c] * chain_len, q, [CHAIN["m"]] * chain_len, bonds, angles)
    bld.add_waters(o_pos, rng, t_o, t_h)
    sigma = [CHAIN["sigma"], WATER_O["sigma"], WATER_H["sigma"]]
    eps = [CHAIN["eps"], WATER_O["eps"], WATER_H["eps"]]
    sys, pos = bld.finish(box, sigma, eps, rc=rc, eps_rf=eps_rf,
                          name=f"chains{n_chains}x{chain_len}_water{n_waters}")
    return sys, pos


def make_path(base: np.ndarray, n_beads: int, seed: int, std: float = 0.01) -> np.ndarray:
    """N beads = base + independent N(0, std) displacements, rounded to float32 once."""
    rng = np.random.default_rng(seed)
    noise = rng.normal(0.0, std, (n_beads,) + base.shape)
    return (base[None, :, :] + noise).astype(np.float32)


def nearest_group(pos: np.ndarray, box: np.ndarray, center: np.ndarray, k: int) -> np.ndarray:
    d = pos - center
    d -= box * np.round(d / box)
    return np.sort(np.argsort(np.einsum("ij,ij->i", d, d), kind="stable")[:k]).astype(np.int32)


# ----------------------------------------------------------------------------------------
# the five workloads

UNEVEN_BEADS = (24, 40, 64, 96, 128, 160, 200, 256)


def config(k: int, n_beads: int | None = None, seed: int | None = None, base=None) -> Workload:
    """Workload k (1..5).  `n_beads` overrides the bead count of every path; `base` (Q x 3)
    replaces the generated base structure (for example a relaxed copy of it) before the beads
    are drawn around it.  The base structure in use is kept in system.extra["base"]."""
    s = 1000 + k if seed is None else seed
    w = _config(k, n_beads, s, base)
    return w


def _config(k: int, n_beads, s: int, base) -> Workload:
    def pick(pos):
        return pos if base is None else np.asarray(base, np.float64).reshape(pos.shape)
    if k == 1:
        sys, pos = lj_fcc()
        pos = pick(pos)
        sys.name = "cfg1_lj256"
        N = 16 if n_beads is None else n_beads
        w = Workload(sys, [make_path(pos, N, s)], precision="fp64", fd_h=1e-5, label="cfg1")
        w.system.extra["base"] = pos
        return w
    if k == 2:
        sys, pos = water_box(1000, rc=0.9, seed=s)
        pos = pick(pos)
        sys.name = "cfg2_water1000"
        sys.extra["base"] = pos
        N = 64 if n_beads is None else n_beads
        return Workload(sys, [make_path(pos, N, s + 100)], label="cfg2")
    if k == 3:
        sys, pos = water_box(8000, rc=1.0, seed=s)
        pos = pick(pos)
        sys.name = "cfg3_water8000"
        sys.extra["base"] = pos
        N = 128 if n_beads is None else n_beads
        return Workload(sys, [make_path(pos, N, s + 100)], label="cfg3")
    if k == 4:
        sys, pos = water_box(3333, rc=1.0, seed=s, n_ions=1)
        pos = pick(pos)
        sys.name = "cfg4_water3333_ion"
        sys.extra["base"] = pos
        beads = UNEVEN_BEADS if n_beads is None else (n_beads,) * len(UNEVEN_BEADS)
        paths = [make_path(pos, n, s + 100 + p) for p, n in enumerate(beads)]
        rng = np.random.default_rng(s + 7)
        ca, cb = rng.random(3) * sys.box, rng.random(3) * sys.box
        ga = nearest_group(pos, sys.box, ca, 8)
        gb = nearest_group(pos, sys.box, cb, 8)
        return Workload(sys, paths, cv_groups=(ga, gb),
                        bias=dict(height=1.0, width=0.05), label="cfg4")
    if k == 5:
        sys, pos = chains_and_water(seed=s)
        pos = pick(pos)
        sys.name = "cfg5_chains_water150k"
        sys.extra["base"] = pos
        N = 64 if n_beads is None else n_beads
        return Workload(sys, [make_path(pos, N, s + 100)], label="cfg5")
    raise ValueError(f"no workload {k}")
